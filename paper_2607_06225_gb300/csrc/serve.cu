// serve.cu -- continuous batching of single-pair requests (filtr_serve_*).
//
// The server owns `lanes`: each lane is a context (own workspace and stream),
// a device I/O buffer, pinned host staging and a host thread.  Submitted
// requests (host copies, codes checked on submit) wait in a FIFO queue.
// Whenever a lane is free, its thread forms a micro-batch from the oldest
// request and the following queued requests with identical parameters and the
// same cost class, as far as the lane's memory allows (sequences + results +
// CIGAR + traceback + staging bytes), copies it in, launches the batched
// alignment on the lane's stream and waits for its event.  Lanes run
// concurrently, so requests that arrive while others are on the GPU start as
// soon as a lane frees up and overlap with them on the device; results move to
// per-ticket host storage and waiters are woken.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "filtr_ctx.h"
#include "k_xdrop_layout.h"
#include "plan.h"

namespace filtr {
namespace {

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Req {
  uint64_t ticket = 0;
  filtr_params p{};
  ScoreParams sp{};
  int8_t subst[MAX_ALPHA * MAX_ALPHA];
  std::vector<uint8_t> q, r;
  uint64_t bytes = 0;   // lane memory this request needs
  uint64_t io = 0;      // of which in the lane's I/O buffer
  uint64_t cells = 0;
  bool big = false;     // runs alone (on the intra-pair kernel unless X-drop)
  int cls = 0;          // cost class: requests batch only within a factor of 4 in cells
  uint64_t t_submit = 0, t_launch = 0, t_done = 0;
  int state = 0;        // 0 queued, 1 running, 2 done
  filtr_status err = FILTR_OK;
  filtr_result res{};
  std::vector<uint32_t> cigar;
};

struct Lane {
  Ctx *ctx = nullptr;
  char *d_io = nullptr;
  size_t io_bytes = 0;
  char *h_io = nullptr;   // pinned, same size as d_io
  cudaEvent_t done = nullptr;
  bool busy = false;
  std::vector<Req *> batch;
  size_t res_off = 0, cig_off = 0;  // inside the I/O buffer
  uint64_t cig_cap = 0;
};

// A request above BIG_CELLS runs alone: one warp would take it tens of
// milliseconds (every request of its micro-batch would wait that long), while
// the intra-pair kernel spreads its row strips over as many warps.
constexpr uint64_t BIG_CELLS = 1ull << 22;
// Micro-batches hold requests of one cost class (cells within a factor of 4),
// so a short request never waits for a long one launched with it.
inline int cost_class(uint64_t cells) {
  int b = 0;
  while (cells >= 4 && b < 31) {
    cells >>= 2;
    ++b;
  }
  return b;
}

}  // namespace

struct Server {
  Ctx *parent = nullptr;
  size_t budget = 0;
  std::vector<Lane> lanes;
  std::vector<std::thread> workers;  // one per lane
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req *> queue;
  std::unordered_map<uint64_t, Req *> table;
  uint64_t next_ticket = 1;
  bool stop = false;
  size_t lane_capacity = 0;   // bytes a micro-batch may use on one lane
  size_t lane_io = 0;         // of which in the lane's I/O buffer
  size_t max_queue = 1 << 20;
  filtr_status fatal = FILTR_OK;
  std::string fatal_msg;
};

namespace {

// bytes one request needs on a lane: I/O (codes, offsets, lengths, result,
// CIGAR) plus workspace (traceback, CIGAR staging, strip buffer share)
uint64_t request_bytes(const ScoreParams &sp, uint32_t M, uint32_t N) {
  uint64_t b = (uint64_t)M + N + 8 * 2 + 4 * 2 + sizeof(filtr_result) + 4ull * (M + N + 1) + 256;
  if (sp.traceback) {
    b += 4ull * (M + N + 1);
    if (sp.use_xdrop)
      b += 4 * xd_tb_words(M, N, 4, 8);  // room for one widened rerun
    else if (M && N)
      b += 4 * full_tb_words(M, N, full_rows_per_lane(M, N), sp);
  }
  b += 64ull * 1024 + 16ull * (N + 2) * 64;  // per-call fixed parts and strip buffers, generous
  return b;
}

bool same_params(const Req *a, const Req *b) {
  return memcmp(&a->sp, &b->sp, sizeof(ScoreParams)) == 0 && a->big == b->big && a->cls == b->cls;
}

// Launch one micro-batch on a free lane (called with the server lock released).
filtr_status launch_batch(Server *S, Lane &L) {
  std::vector<Req *> &B = L.batch;
  const uint32_t n = (uint32_t)B.size();
  uint64_t qbytes = 0, rbytes = 0, ops = 0;
  for (Req *r : B) {
    qbytes += r->q.size();
    rbytes += r->r.size();
    ops += r->q.size() + r->r.size();
  }
  auto al = [](uint64_t x) { return (x + 255) / 256 * 256; };
  size_t off = 0;
  const size_t o_q = off;
  off += al(qbytes + 1);
  const size_t o_r = off;
  off += al(rbytes + 1);
  const size_t o_qo = off;
  off += al(8ull * n);
  const size_t o_ro = off;
  off += al(8ull * n);
  const size_t o_ql = off;
  off += al(4ull * n);
  const size_t o_rl = off;
  off += al(4ull * n);
  const size_t o_res = off;
  off += al(sizeof(filtr_result) * n);
  const size_t o_cig = off;
  off += al(4 * (ops + 1));
  if (off > L.io_bytes) {
    set_error("micro-batch I/O (%zu bytes) exceeds the lane buffer", off);
    return FILTR_ERR_NOMEM;
  }
  char *h = L.h_io;
  uint64_t *qo = reinterpret_cast<uint64_t *>(h + o_qo), *ro = reinterpret_cast<uint64_t *>(h + o_ro);
  uint32_t *ql = reinterpret_cast<uint32_t *>(h + o_ql), *rl = reinterpret_cast<uint32_t *>(h + o_rl);
  uint64_t aq = 0, ar = 0;
  for (uint32_t t = 0; t < n; ++t) {
    Req *r = B[t];
    memcpy(h + o_q + aq, r->q.data(), r->q.size());
    memcpy(h + o_r + ar, r->r.data(), r->r.size());
    qo[t] = aq;
    ro[t] = ar;
    ql[t] = (uint32_t)r->q.size();
    rl[t] = (uint32_t)r->r.size();
    aq += r->q.size();
    ar += r->r.size();
  }
  cudaStream_t st = L.ctx->own_stream;
  cudaError_t e = cudaMemcpyAsync(L.d_io, h, o_res, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "serve: host-to-device copy");
  BatchDev b{reinterpret_cast<uint8_t *>(L.d_io + o_q), reinterpret_cast<uint8_t *>(L.d_io + o_r),
             reinterpret_cast<uint64_t *>(L.d_io + o_qo), reinterpret_cast<uint64_t *>(L.d_io + o_ro),
             reinterpret_cast<uint32_t *>(L.d_io + o_ql), reinterpret_cast<uint32_t *>(L.d_io + o_rl)};
  filtr_result *dres = reinterpret_cast<filtr_result *>(L.d_io + o_res);
  uint32_t *dcig = reinterpret_cast<uint32_t *>(L.d_io + o_cig);
  filtr_status rc;
  if (n == 1 && B[0]->big && !B[0]->sp.use_xdrop && B[0]->q.size() > 1024 && !B[0]->r.empty()) {
    // a large request: every SM on it (intra-pair strips) instead of one warp
    rc = long_pair_async(L.ctx, B[0]->sp, &B[0]->p, b.q_seq, (uint32_t)B[0]->q.size(), b.r_seq,
                         (uint32_t)B[0]->r.size(), dres, B[0]->sp.traceback ? dcig : nullptr,
                         B[0]->sp.traceback ? ops + 1 : 0, st);
  } else {
    rc = align_batch_impl(L.ctx, &B[0]->p, n, b, dres, B[0]->sp.traceback ? dcig : nullptr,
                          B[0]->sp.traceback ? ops + 1 : 0, st, false, ql, rl, true);
  }
  if (rc != FILTR_OK) return rc;
  e = cudaMemcpyAsync(h + o_res, L.d_io + o_res, sizeof(filtr_result) * n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && B[0]->sp.traceback)
    e = cudaMemcpyAsync(h + o_cig, L.d_io + o_cig, 4 * (ops + 1), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaEventRecord(L.done, st);
  if (e != cudaSuccess) return cuda_fail(e, "serve: device-to-host copy");
  L.res_off = o_res;
  L.cig_off = o_cig;
  L.cig_cap = ops + 1;
  return FILTR_OK;
}

void finish_batch(Lane &L, uint64_t t) {
  const filtr_result *res = reinterpret_cast<const filtr_result *>(L.h_io + L.res_off);
  const uint32_t *cig = reinterpret_cast<const uint32_t *>(L.h_io + L.cig_off);
  for (size_t k = 0; k < L.batch.size(); ++k) {
    Req *r = L.batch[k];
    r->res = res[k];
    if (r->sp.traceback && r->res.cigar_len)
      r->cigar.assign(cig + r->res.cigar_off, cig + r->res.cigar_off + r->res.cigar_len);
    r->res.cigar_off = 0;
    r->t_done = t;
    r->state = 2;
  }
  L.batch.clear();
  L.busy = false;
}

// One host thread per lane: it takes the next micro-batch from the shared
// queue when its lane is free, launches it and waits for it.  A batch whose
// host code must wait for the device (the X-drop sweep reads back the pairs
// that outgrew their window) then holds up only its own lane.
void lane_main(Server *S, Lane *Lp) {
  Lane &L = *Lp;
  cudaSetDevice(S->parent->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    S->cv_work.wait(lk, [&] { return S->stop || !S->queue.empty(); });
    if (S->stop) break;
    Req *head = S->queue.front();
    uint64_t used = 0, used_io = 0;
    std::vector<Req *> pick;
    for (auto it = S->queue.begin(); it != S->queue.end();) {
      Req *r = *it;
      if (same_params(head, r) &&
          (pick.empty() || (used + r->bytes <= S->lane_capacity && used_io + r->io <= S->lane_io)) &&
          pick.size() < 65536) {
        used += r->bytes;
        used_io += r->io;
        pick.push_back(r);
        it = S->queue.erase(it);
        if (r->big) break;  // big requests run alone
      } else {
        ++it;
      }
    }
    const uint64_t t = now_ns();
    for (Req *r : pick) {
      r->state = 1;
      r->t_launch = t;
    }
    L.batch = pick;
    L.busy = true;
    if (!S->queue.empty()) S->cv_work.notify_one();  // another lane may take the rest
    lk.unlock();
    filtr_status rc = launch_batch(S, L);
    cudaError_t e = cudaSuccess;
    if (rc == FILTR_OK) e = cudaEventSynchronize(L.done);
    lk.lock();
    if (rc == FILTR_OK && e == cudaSuccess) {
      finish_batch(L, now_ns());
    } else {
      if (rc == FILTR_OK) {
        rc = FILTR_ERR_CUDA;
        S->fatal = FILTR_ERR_CUDA;
        S->fatal_msg = cudaGetErrorString(e);
      }
      for (Req *r : L.batch) {
        r->err = rc;
        r->state = 2;
        r->t_done = now_ns();
      }
      L.batch.clear();
      L.busy = false;
    }
    S->cv_done.notify_all();
  }
}

filtr_status take_result(Server *S, Req *r, filtr_result *out, uint32_t *cigar, uint64_t cap,
                         uint64_t *times) {
  if (r->err != FILTR_OK) {
    const filtr_status e = r->err;
    S->table.erase(r->ticket);
    delete r;
    set_error("request failed on the device");
    return e;
  }
  if (out) *out = r->res;
  if (times) {
    times[0] = r->t_submit;
    times[1] = r->t_launch;
    times[2] = r->t_done;
  }
  if (r->cigar.size() > cap) {
    set_error("cigar capacity %llu < %zu ops", (unsigned long long)cap, r->cigar.size());
    return FILTR_ERR_CIGAR_CAP;
  }
  if (cigar && !r->cigar.empty()) memcpy(cigar, r->cigar.data(), r->cigar.size() * 4);
  S->table.erase(r->ticket);
  delete r;
  return FILTR_OK;
}

}  // namespace
}  // namespace filtr

using namespace filtr;

extern "C" {

filtr_status filtr_serve_create(filtr_ctx *ctx, size_t mem_budget, uint32_t max_inflight,
                                filtr_server **out) {
  if (!ctx || !out || max_inflight == 0 || max_inflight > 64) {
    set_error("serve_create: bad arguments");
    return FILTR_ERR_INVALID;
  }
  *out = nullptr;
  Ctx *parent = reinterpret_cast<Ctx *>(ctx);
  Server *S = new (std::nothrow) Server();
  if (!S) return FILTR_ERR_NOMEM;
  S->parent = parent;
  S->budget = mem_budget;
  // per lane: a small I/O buffer (codes, results, CIGARs) and a workspace for
  // the traceback; one request may use most of a lane, a micro-batch as much
  const size_t per_lane = mem_budget / max_inflight;
  const size_t io = std::max<size_t>(per_lane / 16, 16u << 20);
  if (per_lane < io + (64u << 20)) {
    delete S;
    set_error("serve_create: budget too small (%zu bytes per lane)", per_lane);
    return FILTR_ERR_INVALID;
  }
  const size_t ws = per_lane - io;
  S->lane_capacity = ws / 10 * 8;
  S->lane_io = io - 4096;
  S->lanes.resize(max_inflight);
  cudaSetDevice(parent->device);
  for (Lane &L : S->lanes) {
    filtr_status rc = ctx_new(parent->device, ws, &L.ctx);
    cudaError_t e = cudaSuccess;
    if (rc == FILTR_OK) e = cudaMalloc(&L.d_io, io);
    if (rc == FILTR_OK && e == cudaSuccess) e = cudaHostAlloc(&L.h_io, io, cudaHostAllocDefault);
    if (rc == FILTR_OK && e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
    if (rc != FILTR_OK || e != cudaSuccess) {
      cudaGetLastError();
      for (Lane &M : S->lanes) {
        if (M.ctx) ctx_delete(M.ctx);
        if (M.d_io) cudaFree(M.d_io);
        if (M.h_io) cudaFreeHost(M.h_io);
        if (M.done) cudaEventDestroy(M.done);
      }
      delete S;
      set_error("serve_create: lane allocation failed");
      return FILTR_ERR_NOMEM;
    }
    L.io_bytes = io;
  }
  for (Lane &L : S->lanes) S->workers.emplace_back(lane_main, S, &L);
  *out = reinterpret_cast<filtr_server *>(S);
  return FILTR_OK;
}

filtr_status filtr_serve_submit(filtr_server *srv, const filtr_params *params, const uint8_t *q,
                                uint32_t M, const uint8_t *r, uint32_t N, uint64_t *ticket) {
  if (!srv || !ticket || (M && !q) || (N && !r)) {
    set_error("serve_submit: NULL argument");
    return FILTR_ERR_INVALID;
  }
  Server *S = reinterpret_cast<Server *>(srv);
  Req *R = new (std::nothrow) Req();
  if (!R) return FILTR_ERR_NOMEM;
  filtr_status rc = to_score_params(params, &R->sp);
  if (rc != FILTR_OK) {
    delete R;
    return rc;
  }
  for (uint32_t i = 0; i < M; ++i)
    if (q[i] >= R->sp.alphabet) {
      delete R;
      set_error("serve_submit: query code >= alphabet");
      return FILTR_ERR_INVALID;
    }
  for (uint32_t j = 0; j < N; ++j)
    if (r[j] >= R->sp.alphabet) {
      delete R;
      set_error("serve_submit: reference code >= alphabet");
      return FILTR_ERR_INVALID;
    }
  R->p = *params;
  memcpy(R->subst, params->subst, (size_t)params->alphabet * params->alphabet);
  R->p.subst = R->subst;
  R->q.assign(q, q + M);
  R->r.assign(r, r + N);
  R->bytes = request_bytes(R->sp, M, N);
  R->io = 256 * 8 + 2ull * (M + N) + 4ull * (M + N + 1) + 64;
  R->cells = band_cells(M, N, R->sp);
  R->big = R->cells > BIG_CELLS;
  R->cls = cost_class(R->cells);
  std::lock_guard<std::mutex> lk(S->mu);
  if (R->bytes > S->lane_capacity || R->io > S->lane_io || S->queue.size() >= S->max_queue ||
      S->stop) {
    delete R;
    set_error("serve_submit: request exceeds the lane budget or the queue is full");
    return FILTR_ERR_BUSY;
  }
  R->ticket = S->next_ticket++;
  R->t_submit = now_ns();
  S->table[R->ticket] = R;
  S->queue.push_back(R);
  *ticket = R->ticket;
  S->cv_work.notify_one();
  return FILTR_OK;
}

filtr_status filtr_serve_poll(filtr_server *srv, uint64_t ticket, filtr_result *out, uint32_t *cigar,
                              uint64_t cap, uint64_t *times_ns) {
  if (!srv) return FILTR_ERR_INVALID;
  Server *S = reinterpret_cast<Server *>(srv);
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->table.find(ticket);
  if (it == S->table.end()) {
    set_error("serve_poll: unknown ticket");
    return FILTR_ERR_INVALID;
  }
  if (it->second->state != 2) return FILTR_ERR_BUSY;
  return take_result(S, it->second, out, cigar, cap, times_ns);
}

filtr_status filtr_serve_wait(filtr_server *srv, uint64_t ticket, int64_t timeout_us,
                              filtr_result *out, uint32_t *cigar, uint64_t cap, uint64_t *times_ns) {
  if (!srv) return FILTR_ERR_INVALID;
  Server *S = reinterpret_cast<Server *>(srv);
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->table.find(ticket);
  if (it == S->table.end()) {
    set_error("serve_wait: unknown ticket");
    return FILTR_ERR_INVALID;
  }
  Req *R = it->second;
  auto ready = [&] { return R->state == 2; };
  if (timeout_us < 0) {
    S->cv_done.wait(lk, ready);
  } else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready)) {
    set_error("serve_wait: timed out");
    return FILTR_ERR_TIMEOUT;
  }
  return take_result(S, R, out, cigar, cap, times_ns);
}

filtr_status filtr_serve_destroy(filtr_server *srv) {
  if (!srv) return FILTR_OK;
  Server *S = reinterpret_cast<Server *>(srv);
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    // queued requests that never launched are dropped
    for (Req *r : S->queue) {
      S->table.erase(r->ticket);
      delete r;
    }
    S->queue.clear();
  }
  S->cv_work.notify_all();
  for (std::thread &w : S->workers)
    if (w.joinable()) w.join();
  for (auto &kv : S->table) delete kv.second;
  for (Lane &L : S->lanes) {
    if (L.ctx) ctx_delete(L.ctx);
    if (L.d_io) cudaFree(L.d_io);
    if (L.h_io) cudaFreeHost(L.h_io);
    if (L.done) cudaEventDestroy(L.done);
  }
  delete S;
  return FILTR_OK;
}

}  // extern "C"
