/* filtr.h -- C ABI of the GB300 pairwise-alignment library.
 *
 * The library evaluates the pairwise sequence-alignment recurrence of
 * "Compiling Bioinformatics Recurrences" (FILTR): Needleman-Wunsch global and
 * Smith-Waterman local alignment (Sec. 1, Sec. 2 edit-distance recurrence), with
 * linear or affine (Gotoh H/E/F, Table 1 "Sequence Alignment") gap costs, exact
 * integer scores, under the pruning rules of Sec. 7 -- a static band
 * (Sec. 7.1 prune axis lo <= diag(i,j) <= hi) and X-drop (Sec. 5.2 conditional
 * definition with the diag_lo / diag_hi domain recurrences, Sec. 7.2) -- and
 * returns score, end coordinates and the traceback as a SAM/BAM CIGAR.  Beside
 * it: Table 1's own M/I/D gap form (FILTR_AFFINE_MID), a running-maximum X-drop
 * threshold (FILTR_PRUNE_XDROP_RUNNING), edit distance by the search traversal
 * of Sec. 6.3 with WFA-Adapt (filtr_search_batch), and Nussinov RNA folding with
 * X-drop transferred to it (Sec. 9.5, filtr_fold_batch).
 *
 * Conventions shared by every entry point
 *   - q is the query (length M, rows i = 1..M), r the reference (length N,
 *     columns j = 1..N); diag(i,j) = j - i, antidiagonal k = i + j (Sec. 6.2).
 *   - Residues are small integer codes, one per byte: DNA 0..3 (A C G T),
 *     protein 0..19.  A code >= the alphabet size is rejected.
 *   - A gap of length L costs gap_open + L*gap_extend (affine) or L*gap_extend
 *     (linear).  E is the horizontal gap (consumes the reference, CIGAR 'D'),
 *     F the vertical gap (consumes the query, CIGAR 'I').
 *   - Ties: H takes the diagonal, then E, then F; E and F prefer opening over
 *     extending; a local H of 0 ends the traceback; the best cell is the largest
 *     H, then the smallest i, then the smallest j.
 *   - Band: with FILTR_PRUNE_BAND the computed cells satisfy lo <= j-i <= hi
 *     where lo = min(0, N-M) - band and hi = max(0, N-M) + band (the band is
 *     widened so it holds both corners); with FILTR_PRUNE_BAND_LITERAL it is
 *     -band <= j-i <= band exactly, and a global alignment whose corner falls
 *     outside reports FILTR_ST_UNREACHABLE.
 *   - X-drop: a cell on antidiagonal k is pruned when H < best(k-1) - xdrop,
 *     best(k-1) being the largest unpruned H of antidiagonal k-1; antidiagonal
 *     k+1 covers the diagonals [lo_k - 1, hi_k + 1] spanned by the unpruned
 *     cells of k; the sweep stops at the first antidiagonal with no unpruned
 *     cell.  A global alignment that does not reach (M,N) reports
 *     FILTR_ST_DROPPED with the best unpruned cell as its end.
 *   - Z-drop (Sec. 9.3): as X-drop, with a cell pruned when
 *     best(k-1) - H > xdrop + |(j - i) - d_best(k-1)|, d_best(k-1) the diagonal
 *     of antidiagonal k-1's best cell (largest H, then smallest i).  With
 *     FILTR_PRUNE_XDROP_RUNNING, best(k-1) becomes the best of every antidiagonal
 *     up to k-1 (and d_best the diagonal where it was first reached).
 *   - CIGAR ops are BAM uint32 words  (len << 4) | op  with op 7 '=', 8 'X',
 *     1 'I', 2 'D'.
 *   - Errors: every function returns a filtr_status; nothing aborts and no
 *     kernel traps.  filtr_last_error() gives a message for the calling thread.
 *   - Streams: `stream` is a cudaStream_t (NULL = the legacy default stream).
 *     Device outputs are complete when the stream reaches that point.
 */
#ifndef FILTR_H
#define FILTR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FILTR_OK = 0,
  FILTR_ERR_INVALID = -1,     /* bad argument; nothing was launched */
  FILTR_ERR_NOMEM = -2,       /* a device or host allocation failed */
  FILTR_ERR_CUDA = -3,        /* a CUDA call failed (message in filtr_last_error) */
  FILTR_ERR_TIMEOUT = -4,     /* a bounded device wait or serve wait ran out */
  FILTR_ERR_BUSY = -5,        /* serve: queue full, or result not ready yet */
  FILTR_ERR_CIGAR_CAP = -6,   /* cigar buffer too small; results carry the lengths needed */
  FILTR_ERR_UNSUPPORTED = -7  /* a size or combination this build does not handle */
} filtr_status;

enum { FILTR_GLOBAL = 0, FILTR_LOCAL = 1 };
enum { FILTR_ALPHA_DNA = 4, FILTR_ALPHA_PROTEIN = 20 };
enum { FILTR_PRUNE_BAND = 1u, FILTR_PRUNE_XDROP = 2u, FILTR_PRUNE_BAND_LITERAL = 4u,
       FILTR_PRUNE_ZDROP = 8u,          /* XDROP and ZDROP exclude each other */
       FILTR_PRUNE_XDROP_RUNNING = 16u  /* with XDROP or ZDROP: the threshold follows the
                                           best score of every antidiagonal so far (a running
                                           maximum, Sec. 9.3's "best score seen so far")
                                           instead of antidiagonal k-1's; for Z-drop the
                                           reference diagonal is that of the antidiagonal that
                                           first reached the running best */ };
enum { FILTR_PREC_AUTO = 0, FILTR_PREC_I32 = 1, FILTR_PREC_I16X2 = 2 };
enum { FILTR_XDROP_INF = 0x7fffffff };

/* per-pair outcome in filtr_result.status */
enum {
  FILTR_ST_OK = 0,
  FILTR_ST_DROPPED = 1,     /* X-drop stopped before (M,N) (global) */
  FILTR_ST_UNREACHABLE = 2, /* literal band excludes (M,N) (global) */
  FILTR_ST_EMPTY = 3,       /* local best score is 0: empty alignment */
  FILTR_ST_TOO_WIDE = 4,    /* X-drop region wider than the kernel window (see filtr_align_batch) */
  FILTR_ST_TIMEOUT = 5      /* a bounded wait of the intra-pair kernel ran out (no result) */
};

/* Table 1's own affine form: M(i,j) = max(M, I, D)(i-1, j-1) + s, I and D open
 * from M only (o + e) and extend themselves (e), so an insertion never touches a
 * deletion (the Gotoh H/E/F form, affine = 1, opens gaps from H = max(M, I, D)).
 * It runs on the antidiagonal sweep: with FILTR_PRUNE_XDROP (running or not),
 * the widened band, or no pruning (no threshold; a pair whose live antidiagonal
 * outgrows 8192 cells reports FILTR_ST_TOO_WIDE).  Not with Z-drop, the literal
 * band, filtr_align_long or filtr_graph_* (FILTR_ERR_UNSUPPORTED). */
#define FILTR_AFFINE_MID 2

typedef struct {
  int32_t mode;          /* FILTR_GLOBAL or FILTR_LOCAL */
  int32_t alphabet;      /* FILTR_ALPHA_DNA or FILTR_ALPHA_PROTEIN */
  int32_t affine;        /* 1: Gotoh H/E/F; 0: linear gap (gap_open ignored);
                            FILTR_AFFINE_MID: Table 1's M/I/D form (see below) */
  int32_t gap_open;      /* >= 0 */
  int32_t gap_extend;    /* >= 0 */
  const int8_t *subst;   /* HOST pointer: alphabet*alphabet scores, subst[q_code*alphabet + r_code];
                            copied during the call; need not be symmetric */
  uint32_t prune;        /* OR of FILTR_PRUNE_* (0 = full matrix) */
  int32_t band;          /* band half-width >= 0 (used with FILTR_PRUNE_BAND) */
  int32_t xdrop;         /* X (or Z) >= 0, or FILTR_XDROP_INF (with FILTR_PRUNE_XDROP / ZDROP) */
  int32_t traceback;     /* 0: score and end cell only; 1: also begin cell and CIGAR */
  int32_t precision;     /* FILTR_PREC_*: a speed choice only; results are identical */
} filtr_params;

typedef struct {
  int32_t score;
  int32_t q_begin, q_end;  /* query residues [q_begin, q_end); q_end = i of the end cell */
  int32_t r_begin, r_end;  /* reference residues [r_begin, r_end); r_end = j of the end cell */
  int32_t status;          /* FILTR_ST_* */
  uint32_t cigar_len;      /* ops of this pair (needed length when the call returned CIGAR_CAP) */
  uint32_t reserved;
  uint64_t cigar_off;      /* first op of this pair in the caller's cigar buffer */
  uint64_t cells;          /* cells (i >= 1, j >= 1) whose recurrence was evaluated, pruned or not */
} filtr_result;            /* 48 bytes.  Without traceback, q_begin = r_begin = -1 for local
                              alignments (unknown) and 0 for global ones; cigar_len = 0. */

typedef struct filtr_ctx filtr_ctx;
typedef struct filtr_server filtr_server;

/* Thread-local message describing the last error of this thread (never NULL). */
const char *filtr_last_error(void);

/* Library version string. */
const char *filtr_version(void);

/* Check a parameter block on the host (no device work).  FILTR_OK or
 * FILTR_ERR_INVALID (negative penalties, unknown mode / alphabet / precision,
 * negative band or xdrop, NULL subst, a linear gap with a band, ...). */
filtr_status filtr_params_check(const filtr_params *params);

/* Create a context on `device`.  The context owns its device workspace
 * (workspace_bytes; 0 picks 8 GiB, capped at half the free device memory),
 * pinned host staging and streams.  One context serves one host thread at a
 * time.  *out receives the context or NULL. */
filtr_status filtr_ctx_create(int device, size_t workspace_bytes, filtr_ctx **out);
filtr_status filtr_ctx_destroy(filtr_ctx *ctx);

/* Pack step (Sec. 2's residue alphabets): validate n residue codes at `codes`
 * (DEVICE, 16-byte aligned: each thread reads 16 codes with one vector load)
 * against `alphabet` and write them packed at `packed` (DEVICE, 4-byte aligned,
 * ceil(n*bits/32) uint32 words, bits = 2 for DNA, 8 for protein; residue t
 * sits at bits [bits*(t % per_word), ...) of word t / per_word; a DNA code
 * keeps its two low bits).  *bad_out (DEVICE, one uint32, not cleared here)
 * gains the number of codes >= alphabet.  Stream ordered; no synchronisation.
 * FILTR_ERR_INVALID for a bad alphabet, a NULL or misaligned pointer. */
filtr_status filtr_pack(const uint8_t *codes, uint64_t n, int32_t alphabet, uint32_t *packed,
                        uint32_t *bad_out, void *stream);

/* Align n_pairs independent pairs in one batched call (Sec. 2 recurrence under
 * the Sec. 7 pruning rules).
 *   q_seq / r_seq : DEVICE, residue codes, one byte each, pairs concatenated
 *   q_off / r_off : DEVICE, uint64 start of each pair's sequence
 *   q_len / r_len : DEVICE, uint32 lengths (0 allowed)
 *   out           : DEVICE, n_pairs filtr_result
 *   cigar         : DEVICE, cigar_cap uint32 ops (may be NULL when traceback = 0)
 * The call reads the lengths back to the host once (a short synchronisation on
 * `stream`) to plan length buckets, traceback waves and kernel shapes; the rest
 * is stream ordered.  Pairs of one call share the params.  The CIGARs are laid
 * out in pair order; if the total exceeds cigar_cap the call returns
 * FILTR_ERR_CIGAR_CAP after the stream completes and each result carries its
 * length.  Band and X-drop pairs whose live region outgrows the widest kernel
 * window (8192 cells on one antidiagonal) get FILTR_ST_TOO_WIDE.  Returns FILTR_ERR_INVALID
 * before any launch for bad params or codes, FILTR_ERR_UNSUPPORTED when scores
 * could reach 2^28 in magnitude (largest |substitution score| x shorter side +
 * 3 x open + extend x (longest query + longest reference)) or, for local
 * alignments, largest |substitution score| x shorter side reaches 2^26.
 * params->precision picks the cell width of unbanded, non-X-drop pairs:
 * FILTR_PREC_I16X2 runs every pair whose score range provably fits 15 bits
 * (substitution scores in [-64, 63] and a bound, for its lengths, on every
 * value the recurrence forms) two cells per 32-bit register, FILTR_PREC_I32
 * never does, and
 * FILTR_PREC_AUTO picks per pair by cost (measured ones after filtr_autotune).
 * No pair is ever computed in a width it could overflow, so results do not
 * depend on the choice. */
filtr_status filtr_align_batch(filtr_ctx *ctx, const filtr_params *params, uint32_t n_pairs,
                               const uint8_t *q_seq, const uint64_t *q_off, const uint32_t *q_len,
                               const uint8_t *r_seq, const uint64_t *r_off, const uint32_t *r_len,
                               filtr_result *out, uint32_t *cigar, uint64_t cigar_cap,
                               void *stream);

/* Same as filtr_align_batch with every array in HOST memory (pinned memory
 * gives the fastest copies).  The call copies the inputs to the device, aligns
 * and copies results and CIGARs back; it returns when they are in host memory. */
filtr_status filtr_align_batch_host(filtr_ctx *ctx, const filtr_params *params, uint32_t n_pairs,
                                    const uint8_t *q_seq, const uint64_t *q_off,
                                    const uint32_t *q_len, const uint8_t *r_seq,
                                    const uint64_t *r_off, const uint32_t *r_len,
                                    filtr_result *out, uint32_t *cigar, uint64_t cigar_cap);

/* The same batch, one kernel launch per pair with one warp each (the plain
 * per-pair form, kept for comparison).  Arguments as filtr_align_batch;
 * results are identical. */
filtr_status filtr_align_batch_plain(filtr_ctx *ctx, const filtr_params *params,
                                     uint32_t n_pairs, const uint8_t *q_seq,
                                     const uint64_t *q_off, const uint32_t *q_len,
                                     const uint8_t *r_seq, const uint64_t *r_off,
                                     const uint32_t *r_len, filtr_result *out, uint32_t *cigar,
                                     uint64_t cigar_cap, void *stream);

/* Score-only batched alignment that allocates nothing (the paper has no
 * counterpart; this is a deployment variant).  Some callers cannot call
 * cudaMalloc -- code inside a host framework that owns all device memory and
 * forbids further allocation, or latency-critical paths that cannot afford
 * cudaMalloc's implicit device-wide synchronisation.  This entry point needs
 * no context and calls no cudaMalloc, cudaFree or allocating library routine:
 * its scratch (a work-queue counter and one strip buffer per resident warp) is
 * a fixed 32 MiB device array inside the library, which every GPU that loads
 * the library holds until the process exits.
 *   params        : traceback must be 0; full matrix or band (no X-drop)
 *   q_seq .. r_len: DEVICE, as filtr_align_batch;  out: DEVICE, n_pairs results
 *   max_query_len / max_ref_len: the longest query / reference of the batch
 *                   (both >= 1, else FILTR_ERR_INVALID); the strip buffers are
 *                   sized by max_ref_len, so the batch runs on fewer warps as it
 *                   grows, and it is rejected with FILTR_ERR_UNSUPPORTED beyond
 *                   2,097,134 reference residues, at 2^30 query residues, or when
 *                   scores could reach 2^28; a pair longer than the limits it
 *                   was given gets status FILTR_ST_TOO_WIDE (the others are
 *                   computed as usual).
 * Results equal filtr_align_batch's (score, end coordinates, status, cells;
 * q_begin / r_begin as without traceback).  The call validates residue codes
 * and waits for that check on `stream` (FILTR_ERR_INVALID for a bad code):
 * every call copies one word to the host and synchronises `stream`.  It then
 * returns with the alignment queued on `stream`.  The first call on a device
 * looks up the scratch array's device address (cudaGetSymbolAddress) with that
 * device current; make that first call before any stream capture.
 * Every call shares the one array and clears its counters first: calls whose
 * work overlaps on the GPU (other streams, other host threads) race and must
 * be serialised by the caller. */
filtr_status filtr_align_batch_noalloc(const filtr_params *params, uint32_t n_pairs,
                                       const uint8_t *q_seq, const uint64_t *q_off,
                                       const uint32_t *q_len, const uint8_t *r_seq,
                                       const uint64_t *r_off, const uint32_t *r_len,
                                       uint32_t max_query_len, uint32_t max_ref_len,
                                       filtr_result *out, void *stream);

/* Align one long pair with every SM of the device working on it.
 *   q, r : DEVICE codes (M, N up to 2^31-1);  out : DEVICE, one filtr_result;
 *   cigar: DEVICE, cigar_cap ops.
 * X-drop pairs run as one antidiagonal sweep with checkpointed traceback: every
 * `C`-th antidiagonal's state is kept, and the backward pass recomputes one
 * segment at a time, so the traceback memory is bounded by the workspace.
 * Band / full-matrix pairs split the query into row strips of 256 rows, one
 * warp per strip at a time, which hand their bottom rows down through global
 * memory with release/acquire progress words; every wait is bounded and a
 * timeout returns FILTR_ERR_TIMEOUT.  Pairs with M <= 512 or M * N < 2^22
 * run as a one-pair batch instead. */
filtr_status filtr_align_long(filtr_ctx *ctx, const filtr_params *params, const uint8_t *q,
                              uint32_t M, const uint8_t *r, uint32_t N, filtr_result *out,
                              uint32_t *cigar, uint64_t cigar_cap, void *stream);

/* Per-call statistics.  With timing on, filtr_align_batch records CUDA events
 * on its stream around each phase; filtr_ctx_last_stats waits for the last
 * call to finish and returns the device time of each phase (ms), the number of
 * kernel launches the call made, its traceback waves and its evaluated cells
 * as planned (the exact counts are in the results). */
typedef struct {
  double ms_validate;   /* residue validation kernel */
  double ms_forward;    /* forward (cell update) kernels, summed over waves */
  double ms_walk;       /* traceback walks, summed over waves */
  double ms_place;      /* CIGAR offset scan and compaction */
  double ms_total;      /* first to last event of the call */
  uint32_t launches;    /* kernels this library launched for the call */
  uint32_t waves;
  uint64_t cells_planned;
  uint32_t pairs_i16x2; /* pairs that ran in the int16x2 tiled kernel */
  uint32_t device_plan; /* 1: the call was planned on the device, 0: on the host */
  double ms_host_wait;  /* host wall time blocked on the validation and length read-back */
  double ms_host_plan;  /* host wall time from the lengths' arrival to the plan's upload */
  uint64_t cells_i16x2; /* of cells_planned, those of the pairs in the int16x2 tiled kernel */
  uint32_t pairs_xd16;  /* X-drop / Z-drop pairs that ran in the int16x2 antidiagonal sweep */
  uint32_t pairs_xd16_rerun; /* of which, pairs that left its 16-bit range and were rerun in int32 */
} filtr_stats;
filtr_status filtr_ctx_set_timing(filtr_ctx *ctx, int enable);
filtr_status filtr_ctx_last_stats(filtr_ctx *ctx, filtr_stats *out);

/* ---- search traversal: edit distance score-major (Sec. 6.3) ----------------
 * The edit-distance recurrence F(i,j) = min(F(i-1,j-1) + [q_i != r_j],
 * F(i-1,j) + 1, F(i,j-1) + 1) iterated by cost instead of position: wavefront
 * s holds, for each diagonal d = j - i of its domain, the furthest row that s
 * edits reach, from the mismatch, insertion and deletion terms of wavefront s-1
 * (diagonals d, d+1, d-1) followed by a free run of matches; each domain is one
 * diagonal wider on each side than the last, clipped to the matrix, and the
 * search ends at the first s whose wavefront reaches (M, N).  Exact: s is the
 * edit distance.  Options (Sec. 7):
 *   band           : >= 0 restricts the diagonals to
 *                    [min(0, N-M) - band, max(0, N-M) + band] (the band of
 *                    filtr_align_batch, mapped to d as Sec. 7.1 describes);
 *                    < 0: no band.  The result is the best path inside the band.
 *   adapt_min_len  : 0 = exact.  > 0 turns on WFA-Adapt (Sec. 7.2, 9.3): once a
 *   adapt_max_dist   wavefront spans at least adapt_min_len diagonals, its
 *                    bounds move inwards past unreached diagonals and past those
 *                    whose remaining distance max(M - i, N - j) exceeds the
 *                    wavefront's smallest by more than adapt_max_dist; only the
 *                    diagonals left feed the next score.  A heuristic: the
 *                    distance found can exceed the edit distance, its CIGAR
 *                    always costs exactly that distance.
 *   traceback      : 1 = CIGAR ('=' 'X' 'I' 'D').  Walking back from (M, N),
 *                    each score level takes the first of mismatch, insertion,
 *                    deletion that gives its value.
 */
typedef struct {
  int32_t traceback;
  int32_t band;
  int32_t adapt_min_len;
  int32_t adapt_max_dist;
  int32_t alphabet;      /* 0: any byte codes; 4: DNA codes 0..3, held two bits each on
                            chip (sixteen residues per comparison); every code is checked
                            and a code >= 4 fails the call with FILTR_ERR_INVALID */
} filtr_search_params;

/* Edit distance of n_pairs independent pairs by the search traversal.
 *   q_seq / r_seq / offsets / lengths : DEVICE, as filtr_align_batch; codes are
 *       compared for equality only (any byte value).  Each sequence is loaded
 *       in whole 16-byte-aligned blocks, so up to 15 bytes on either side of it
 *       are read (never outside the 16-byte blocks holding its ends).
 *   out   : DEVICE, n_pairs filtr_result: score = minus the distance found (the
 *           unit-cost global alignment score: match 0, mismatch -1, gap 1 per
 *           residue), q_begin = r_begin = 0, q_end = M, r_end = N, status
 *           FILTR_ST_OK, cells = wavefront entries evaluated (the sum over scores
 *           of the domain's width)
 *   cigar : DEVICE, cigar_cap ops (may be NULL without traceback); CIGARs in
 *           pair order, FILTR_ERR_CIGAR_CAP as filtr_align_batch.
 * The call reads the lengths back once (a short synchronisation on `stream`);
 * with traceback it also reads back each pair's wavefront storage (a second
 * synchronisation) and recomputes the pairs with every wavefront kept, in
 * waves that fit the workspace.  FILTR_ERR_INVALID for NULL pointers,
 * negative adapt thresholds, an alphabet other than 0 or 4, or (alphabet 4) a
 * code >= 4; FILTR_ERR_UNSUPPORTED when a pair has
 * M + N > FILTR_SEARCH_MAX_LEN (its sequences are staged in shared memory);
 * FILTR_ERR_NOMEM when one pair's wavefronts do not fit the workspace. */
#define FILTR_SEARCH_MAX_LEN 180000u
filtr_status filtr_search_batch(filtr_ctx *ctx, const filtr_search_params *params,
                                uint32_t n_pairs, const uint8_t *q_seq, const uint64_t *q_off,
                                const uint32_t *q_len, const uint8_t *r_seq,
                                const uint64_t *r_off, const uint32_t *r_len, filtr_result *out,
                                uint32_t *cigar, uint64_t cigar_cap, void *stream);

/* ---- RNA folding with X-drop transferred to it (Sec. 9.5) -----------------
 * Table 1's Nussinov recurrence over the triangle 0 <= i <= j < n:
 *   F(i,j) = max(F(i+1,j), F(i,j-1), F(i+1,j-1) + 1 if i pairs j,
 *                max over i <= m < j of F(i,m) + F(m+1,j)),  F(i,i) = 0,
 * the largest number of nested base pairs, swept span by span (k = j - i).
 * Bases pair as A-U, C-G or G-U (codes A=0 C=1 G=2 U=3) with at least min_loop
 * bases between them.  With use_xdrop, the X-drop rule of alignment is reused
 * on the spans: after the first `warmup` spans (the paper uses 15) a cell is
 * pruned when F < best(k-1) - X, best(k-1) the largest unpruned F of the span
 * before, and span k covers the positions [lo - 1, hi] of the unpruned cells of
 * span k-1; the sweep stops at the first span with nothing unpruned.  The result
 * is F(0, n-1) (FILTR_ST_OK), or, when that cell was pruned or never reached,
 * the best unpruned cell (FILTR_ST_DROPPED: largest F, then longest span, then
 * smallest i) with its fold. */
#define FILTR_FOLD_MAX_LEN 4096u
typedef struct {
  int32_t min_loop;   /* >= 0 */
  int32_t use_xdrop;  /* 1: X-drop on the spans */
  int32_t xdrop;      /* X >= 0 */
  int32_t warmup;     /* spans <= warmup are never pruned; >= 0 */
  int32_t traceback;  /* 1: write the fold to partner */
} filtr_fold_params;

typedef struct {
  int32_t score;        /* base pairs: F of the end cell */
  int32_t i_end, j_end; /* the end cell (0, n-1), or the best unpruned one when DROPPED */
  int32_t status;       /* FILTR_ST_OK or FILTR_ST_DROPPED */
  uint64_t cells;       /* cells evaluated, span 0 included (n(n+1)/2 unpruned) */
} filtr_fold_result;    /* 24 bytes */

/* Fold n_seqs RNAs.
 *   seq / off / len : DEVICE, codes (one byte each, 0..3), uint64 starts, uint32
 *                     lengths (<= FILTR_FOLD_MAX_LEN)
 *   out             : DEVICE, n_seqs filtr_fold_result
 *   partner         : DEVICE, int32 per base at the base's own offset (same
 *                     layout as seq): its partner's index within the sequence,
 *                     or -1 (required with traceback, else may be NULL)
 * One synchronisation (codes and lengths); each sequence's triangle
 * (n(n+1)/2 words) lives in the context's workspace, in waves of sequences that
 * fit.  FILTR_ERR_INVALID for NULL pointers, negative parameters or a code >= 4;
 * FILTR_ERR_UNSUPPORTED for a sequence over FILTR_FOLD_MAX_LEN; FILTR_ERR_NOMEM
 * when one triangle does not fit the workspace. */
filtr_status filtr_fold_batch(filtr_ctx *ctx, const filtr_fold_params *params, uint32_t n_seqs,
                              const uint8_t *seq, const uint64_t *off, const uint32_t *len,
                              filtr_fold_result *out, int32_t *partner, void *stream);

/* ---- Captured batch pipeline (CUDA graph) --------------------------------
 * The batched path of filtr_align_batch for tiled batches (full matrix or
 * static band, no X-drop), captured once as a CUDA graph and replayed per batch
 * with no host synchronisation: the residue check, the device plan, one
 * persistent launch per tiled shape, the traceback walks and the CIGAR
 * placement run back to back on the device (the batching pattern of the
 * paper's GPU-side design; the paper itself has no counterpart).  Results are
 * identical to filtr_align_batch's.
 *
 * filtr_graph_create: bounds fixed at creation -- at most max_pairs pairs per
 *   launch, every query and reference at most max_len residues -- and the
 *   graph's own device memory, workspace_bytes in all (capacity-sized plan
 *   arrays, strip buffers and CIGAR staging of max_pairs x (2 max_len + 1)
 *   words, then the traceback area: the rest).  Plans with the context's tuned
 *   shape costs as they are at creation.  Synchronous; allocates.
 *   Errors: FILTR_ERR_INVALID (NULL ctx or out, bad params, zero bounds,
 *   max_len >= 2^30), FILTR_ERR_UNSUPPORTED (X-drop / Z-drop parameters, or
 *   scores that could exceed the int32 range for max_len), FILTR_ERR_NOMEM
 *   (workspace_bytes below the fixed parts), FILTR_ERR_CUDA.
 * filtr_graph_launch: one batch, arguments as filtr_align_batch's (device
 *   pointers); enqueues the graph on stream and returns.  Launches of one graph
 *   share its memory: issue them on one stream (or order them), from one host
 *   thread at a time.  Errors found on the host: FILTR_ERR_INVALID (NULL
 *   graph or pointers, n_pairs > max_pairs), FILTR_ERR_CUDA.  n_pairs = 0
 *   launches nothing.
 * filtr_graph_status: after the stream has finished the last launch, that
 *   launch's outcome: FILTR_OK, FILTR_ERR_INVALID (a residue code >= the
 *   alphabet size, or a sequence longer than max_len: nothing was aligned),
 *   FILTR_ERR_NOMEM (the batch's traceback exceeds the traceback area: nothing
 *   was aligned), FILTR_ERR_CIGAR_CAP (results complete, CIGARs that do not
 *   fit cigar_cap not written), FILTR_ERR_UNSUPPORTED (the plan chose a tile
 *   shape that the graph, which launches only the shapes some pair within its
 *   bounds can take, does not hold: nothing was aligned; not expected).
 * filtr_graph_destroy: waits for the device, frees the graph; NULL is a no-op. */
typedef struct filtr_graph filtr_graph;
filtr_status filtr_graph_create(filtr_ctx *ctx, const filtr_params *params, uint32_t max_pairs,
                                uint32_t max_len, size_t workspace_bytes, filtr_graph **out);
filtr_status filtr_graph_launch(filtr_graph *graph, uint32_t n_pairs, const uint8_t *q_seq,
                                const uint64_t *q_off, const uint32_t *q_len, const uint8_t *r_seq,
                                const uint64_t *r_off, const uint32_t *r_len, filtr_result *out,
                                uint32_t *cigar, uint64_t cigar_cap, void *stream);
filtr_status filtr_graph_status(filtr_graph *graph);
filtr_status filtr_graph_destroy(filtr_graph *graph);

/* Autotuning of the tiled kernel shapes (the paper leaves autotuning to
 * future work, Sec. 11).  Times every tiled shape -- the int32 tile with 32,
 * 24, 16 or 8 rows per lane and, where the parameters allow it, the int16x2
 * tile with any even height from 32 down to 8 -- on calibration batches that fill
 * every resident warp slot of the device three times (pairs of one full strip
 * of query rows by 512 reference residues, random codes), and keeps in ctx the
 * device time per warp step of each shape for this recurrence kind (mode, gap
 * model, traceback, alphabet, band).  Later filtr_align_batch calls of the same
 * kind give each pair the shape whose predicted time, strips x (N + fill
 * steps) x that cost, is smallest.  Results never change: the shapes are
 * bit-exact alternatives.
 *   out: optional; n_shapes (17) entries of rows_per_lane / packed describe the
 *        shapes, always in this order: int32 R = 32, 24, 16, 8, then int16x2
 *        R = 32, 30, 28, ..., 10, 8; ns_per_warp_step is 0 for shapes not
 *        timed (not allowed for these parameters, or too large for the
 *        workspace); entries past n_shapes are 0.
 * With X-drop / Z-drop parameters it tunes the antidiagonal sweep instead:
 * the int16x2 and int32 sweeps at a first group width of 1 and of 2 (windows of
 * 256 and 512 slots; a width-2 window of the int16x2 sweep is one warp of
 * 16-slot threads, of the int32 sweep two warps)
 * each run a batch of related pairs (2048-residue random references, queries
 * with 5% substitutions, 2% insertions, 2% deletions) filling the device twice,
 * and the context keeps, for this recurrence kind (mode, alphabet, traceback,
 * band, Z-drop, running threshold), the candidate with the smallest time per
 * evaluated cell among those that finished at least 99% of the pairs without
 * outgrowing their window; later calls start X-drop pairs at that width and
 * cell width (the int16x2 sweep still only where the threshold leaves room).
 * The report then lists n_shapes = 4 candidates: rows_per_lane = the first
 * group width in warps (1, 1, 2, 2), packed = 1 for the int16x2 sweep (1, 0,
 * 1, 0), ns_per_warp_step = nanoseconds per evaluated cell (0: not run).
 * Synchronous (waits for the context's previous call); uses the workspace.
 * Errors: FILTR_ERR_INVALID (NULL ctx, bad params), FILTR_ERR_NOMEM (the
 * workspace holds no calibration batch), FILTR_ERR_CUDA. */
#define FILTR_TUNE_MAX_SHAPES 24
typedef struct {
  int32_t n_shapes;
  int32_t rows_per_lane[FILTR_TUNE_MAX_SHAPES];
  int32_t packed[FILTR_TUNE_MAX_SHAPES];
  double ns_per_warp_step[FILTR_TUNE_MAX_SHAPES];
} filtr_tune_report;
filtr_status filtr_autotune(filtr_ctx *ctx, const filtr_params *params, filtr_tune_report *out);

/* Install a tune report saved from an earlier filtr_autotune of the same
 * recurrence kind on the same kind of device (no counterpart in the paper):
 * a service restarts with its measured shape costs instead of timing again,
 * and a profiled run plans exactly as an unprofiled one did.  Shapes whose
 * ns_per_warp_step is 0 keep the built-in cost scaled to the given ones.
 * Host only: launches nothing, does not wait for the GPU.
 * With X-drop / Z-drop parameters the report is a sweep report (4 candidates
 * as filtr_autotune lists them) and the fastest timed candidate is installed.
 * Errors: FILTR_ERR_INVALID (NULL ctx or report, bad params, a shape or
 * candidate list other than the one filtr_autotune reports, in its order, a
 * negative or non-finite cost, or no positive cost). */
filtr_status filtr_tune_apply(filtr_ctx *ctx, const filtr_params *params,
                              const filtr_tune_report *report);

/* Measured integer / DPX throughput of this device, used as the cell-update
 * roofline denominator: out[0] = int32 add/max ops per second (all SMs,
 * independent chains), out[1] = __viaddmax_s32 per second, out[2] =
 * __vimax3_s32 per second, out[3] = __viaddmax_s16x2 per second (two lanes per
 * op), out[4] = the SM clock (Hz) the probe ran at, estimated from clock64(). */
filtr_status filtr_probe_int_peak(filtr_ctx *ctx, double out[5]);

/* ---- serving: continuous batching of single-pair requests ------------------
 * Requests are copied into resident device buffers, admitted while their
 * device memory (sequences + DP workspace + traceback bytes) fits mem_budget,
 * grouped by kind and cost class (cells within a factor of 4) into
 * micro-batches and launched on up to max_inflight streams; a micro-batch
 * launches as soon as a stream is free, so requests that arrive while others
 * run overlap with them on the device.  A request above 2^22 cells runs alone,
 * on the intra-pair kernel when it is not X-drop.  Each stream has a host
 * thread owned by the server, which launches its micro-batches and waits for
 * them.  Load the library's kernels eagerly in a serving process
 * (CUDA_MODULE_LOADING=EAGER in the environment before CUDA starts): with lazy
 * loading, the first launch of each kernel waits for the device's running work,
 * and the batches already in flight on the other streams wait with it. */
filtr_status filtr_serve_create(filtr_ctx *ctx, size_t mem_budget, uint32_t max_inflight,
                                filtr_server **out);
/* Queue one pair (HOST pointers, copied before returning).  FILTR_ERR_BUSY if the
 * request alone exceeds the budget or the host queue is full; *ticket
 * identifies the request. */
filtr_status filtr_serve_submit(filtr_server *srv, const filtr_params *params, const uint8_t *q,
                                uint32_t M, const uint8_t *r, uint32_t N, uint64_t *ticket);
/* Non-blocking: FILTR_OK and the result (HOST out, cigar up to cap ops, and if
 * times_ns is not NULL the host monotonic times in ns of submit, launch and
 * completion), or FILTR_ERR_BUSY if not finished.  A retrieved ticket is
 * forgotten; FILTR_ERR_INVALID for an unknown ticket; FILTR_ERR_CIGAR_CAP if
 * cap is too small (out->cigar_len tells the length; the ticket is kept). */
filtr_status filtr_serve_poll(filtr_server *srv, uint64_t ticket, filtr_result *out,
                              uint32_t *cigar, uint64_t cap, uint64_t *times_ns);
/* Blocking variant of poll with a timeout in microseconds (< 0 waits forever);
 * FILTR_ERR_TIMEOUT when it runs out. */
filtr_status filtr_serve_wait(filtr_server *srv, uint64_t ticket, int64_t timeout_us,
                              filtr_result *out, uint32_t *cigar, uint64_t cap,
                              uint64_t *times_ns);
filtr_status filtr_serve_destroy(filtr_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* FILTR_H */
