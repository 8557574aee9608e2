// graph.cu -- filtr_graph: the batched tiled pipeline captured once as a CUDA
// graph and replayed per batch without host synchronisation.
//
// filtr_align_batch synchronises once per call: the host reads the residue
// check and the device plan's totals back before it sizes the workspace and
// launches the forward kernels.  A graph fixes everything that needs: the
// bounds (pairs, sequence length) and the device memory are set at creation,
// every tiled shape's kernel is launched with a persistent grid and takes its
// slice of the order from the device plan, and the per-batch values (sequence
// and output pointers, pair count) live in a device descriptor that the
// graph's first node writes from its kernel arguments, which each launch
// updates.  Checks the host made before (residue codes, lengths within bounds,
// traceback within budget, CIGAR capacity) run as graph nodes: a failed check
// sets the descriptor's abort code, later nodes do nothing, and the code lands
// in a host-mapped word that filtr_graph_status returns once the stream is done.
#include <cmath>
#include <cstddef>
#include <cstring>
#include <vector>

#include "filtr_ctx.h"

namespace filtr {
namespace {

__global__ void k_graph_desc(GraphDesc d, GraphDesc *dst) {
  d.abort = 0;
  *dst = d;
}

// One thread: the checks filtr_align_batch makes on the host.
// One thread: the checks filtr_align_batch makes on the host, and that every
// pair's shape is one the graph launches (shapes_in: bit k for shape k).
__global__ void k_graph_check(const DevPlanState *ps, GraphDesc *gd, uint32_t max_len,
                              unsigned long long tb_cap, unsigned long long stage_cap,
                              uint32_t shapes_in) {
  int32_t code = 0;
  if (ps->bad[0] != 0 || ps->sum.max_m > max_len || ps->sum.max_n > max_len)
    code = FILTR_ERR_INVALID;
  else if (ps->sum.tb_words > tb_cap || ps->sum.stage_words > stage_cap)
    code = FILTR_ERR_NOMEM;
  for (int k = 0; k < SHAPE_TILED && code == 0; ++k)
    if (!(shapes_in >> k & 1u) && ps->sum.count[k] != 0) code = FILTR_ERR_UNSUPPORTED;
  gd->abort = code;
}

// One condition per tiled shape: its conditional node runs the shape's kernel
// only when the device plan gave it pairs (and nothing was aborted).
struct CondArgs {
  cudaGraphConditionalHandle h[SHAPE_TILED];
  int shape[SHAPE_TILED];
  int n;
};
__global__ void k_graph_setcond(const CondArgs c, const DevPlanSummary *sum, const GraphDesc *gd) {
  const bool go = gd->abort == 0;
  for (int i = 0; i < c.n; ++i)  // one thread: no concurrent setters
    cudaGraphSetConditional(c.h[i], (go && sum->count[c.shape[i]] > 0) ? 1u : 0u);
}

__global__ void k_graph_finish(const GraphDesc *gd, const uint64_t *cigar_total, int traceback,
                               int32_t *status) {
  int32_t code = gd->abort;
  if (code == 0 && traceback && *cigar_total > gd->cap) code = FILTR_ERR_CIGAR_CAP;
  *status = code;
}

struct GCarve {
  char *base;
  size_t used = 0;
  template <class T>
  T *take(size_t count) {
    used = (used + 255) / 256 * 256;
    T *p = reinterpret_cast<T *>(base + used);
    used += count * sizeof(T);
    return p;
  }
};

}  // namespace

struct Graph {
  Ctx *ctx = nullptr;
  ScoreParams sp{};
  uint32_t max_pairs = 0, max_len = 0;
  char *mem = nullptr;
  GraphDesc *d_gd = nullptr;
  int32_t *h_status = nullptr;  // host-mapped
  int32_t *d_status = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t desc_node = nullptr;
  cudaKernelNodeParams desc_params{};
};

}  // namespace filtr

using namespace filtr;

namespace {

void graph_free(Graph *g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->h_status) cudaFreeHost(g->h_status);
  if (g->mem) cudaFree(g->mem);
  delete g;
}

// The tiled shapes a graph launches, and each one's persistent grid.
struct ShapeSet {
  int k[SHAPE_TILED];
  int grid[SHAPE_TILED];
  int n = 0;
};
// Shapes choose_shape can give some pair with both lengths at most max_len.
// Within one block of 64 query rows every shape's strip count is fixed and its
// cost is a line in N, so the cheapest shape changes only where two lines
// cross: evaluating the choice at N = 1, N = max_len and beside every crossing
// finds every winner, for pairs that fit 15 bits and for pairs that do not.
// Above 2^20 every allowed shape is kept (the scan would take too long).
void reachable_shapes(const ShapeTable &t, const ScoreParams &sp, uint32_t max_len,
                      bool *reach) {
  for (int k = 0; k < SHAPE_TILED; ++k) reach[k] = false;
  if (max_len > (1u << 20)) {
    for (int i = 0; i < t.n_elig; ++i) reach[t.elig[i]] = true;
    return;
  }
  const uint32_t smax = (max_len + 63) / 64;  // strip counts change every 64 rows
  std::vector<uint32_t> ns;
  for (uint32_t s = 1; s <= smax; ++s) {
    const uint32_t M = std::min<uint32_t>(64 * s, max_len);
    // lines a_k (N + f_k) for this strip count
    double a[SHAPE_TILED];
    for (int i = 0; i < t.n_elig; ++i) {
      const int k = t.elig[i];
      a[k] = (double)strips_of(M, t.R[k]) * t.coef[k];
    }
    ns.assign({1u, max_len});
    for (int i = 0; i < t.n_elig; ++i)
      for (int j = i + 1; j < t.n_elig; ++j) {
        const int k1 = t.elig[i], k2 = t.elig[j];
        if (a[k1] == a[k2]) continue;
        const double x = (a[k2] * t.fill[k2] - a[k1] * t.fill[k1]) / (a[k1] - a[k2]);
        if (!(x > 0 && x < (double)max_len + 1)) continue;
        for (double d : {-1.0, 0.0, 1.0, 2.0}) {
          const double v = std::floor(x) + d;
          if (v >= 1 && v <= max_len) ns.push_back((uint32_t)v);
        }
      }
    for (uint32_t N : ns)
      for (int pk = 0; pk < 2; ++pk) {
        if (pk && t.n_elig_packed == 0) continue;
        const bool packable = pk == 1;
        reach[choose_shape_p(t, packable, packable && sp.precision == FILTR_PREC_I16X2, M, N)] = true;
      }
  }
}

ShapeSet graph_shapes(Ctx *c, const ScoreParams &sp, const ShapeCost *costs, uint32_t max_len) {
  ShapeSet ss;
  const bool pack_ok = !sp.use_band && sp.precision != FILTR_PREC_I32;
  bool reach[SHAPE_TILED];
  reachable_shapes(make_shape_table(costs, sp), sp, max_len, reach);
  for (int k = 0; k < SHAPE_TILED; ++k) {
    if (costs[k].packed && !pack_ok) continue;
    if (!reach[k]) continue;
    const int R = costs[k].R;
    const int bps = c->graph_blocks_per_sm(R, costs[k].packed, sp);
    ss.k[ss.n] = k;
    ss.grid[ss.n] = c->sms * bps;
    ++ss.n;
  }
  return ss;
}

// Capture the pipeline on st into g->graph.  The shapes' kernels sit in
// conditional nodes on parallel branches (each with its own strip buffers and
// queue counter), so a shape the plan leaves empty costs nothing and the
// shapes' tails overlap.  Returns the first error.
cudaError_t capture(Graph *g, const ShapeCost *costs, const ShapeSet &ss, uint64_t tb_words,
                    uint64_t stage_cap, const GCarve &layout_in, cudaStream_t st,
                    cudaStream_t st2) {
  const ScoreParams &sp = g->sp;
  const uint32_t NP = g->max_pairs;
  GCarve cv = layout_in;
  DevPlanState *d_ps = cv.take<DevPlanState>(1);
  uint32_t *d_order = cv.take<uint32_t>(NP);
  TbLayout *d_tbl = cv.take<TbLayout>(NP);
  uint64_t *d_stage_off = cv.take<uint64_t>(NP);
  FwdOut *d_fwd = cv.take<FwdOut>(NP);
  uint64_t *d_offs = cv.take<uint64_t>(NP);
  uint32_t *d_counters = cv.take<uint32_t>(64);
  uint64_t *d_total = cv.take<uint64_t>(4);
  uint16_t *d_pkey = cv.take<uint16_t>(NP);
  uint64_t *d_pwords = cv.take<uint64_t>(NP);
  uint64_t *d_pblk = cv.take<uint64_t>((NP + DEV_PLAN_BLOCK - 1) / DEV_PLAN_BLOCK);
  const uint32_t strip_stride = g->max_len + 2;
  int2 *d_strip[SHAPE_TILED];
  for (int i = 0; i < ss.n; ++i)
    d_strip[i] = cv.take<int2>((size_t)ss.grid[i] * FULL_WARPS * strip_stride);
  uint32_t *d_stage = sp.traceback ? cv.take<uint32_t>(stage_cap) : nullptr;
  uint32_t *d_tb = cv.take<uint32_t>(tb_words);
  uint32_t *d_bad = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(d_ps) +
                                                 offsetof(DevPlanState, bad));

  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  GraphDesc zero{};
  k_graph_desc<<<1, 1, 0, st>>>(zero, g->d_gd);  // the root node: updated per launch
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(d_ps, 0, sizeof(DevPlanState), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_counters, 0, 64 * sizeof(uint32_t), st);
  const BatchDev none{};
  if (e == cudaSuccess) e = launch_validate_pairs(none, NP, sp.alphabet, d_bad, st, g->d_gd);
  DevPlanArgs pa{};
  pa.n = NP;
  pa.sp = sp;
  pa.tab = make_shape_table(costs, sp);
  pa.state = d_ps;
  pa.key = d_pkey;
  pa.words = d_pwords;
  pa.blk = d_pblk;
  pa.order = d_order;
  pa.tbl = d_tbl;
  pa.stage_off = d_stage_off;
  pa.gd = g->d_gd;
  if (e == cudaSuccess) e = launch_plan(pa, st);
  if (e == cudaSuccess) {
    uint32_t shapes_in = 0;
    for (int i = 0; i < ss.n; ++i) shapes_in |= 1u << ss.k[i];
    k_graph_check<<<1, 1, 0, st>>>(d_ps, g->d_gd, g->max_len, (unsigned long long)tb_words,
                                   (unsigned long long)(sp.traceback ? stage_cap : ~0ull),
                                   shapes_in);
    e = cudaGetLastError();
  }
  // conditions, then one conditional branch per shape
  cudaGraph_t cg = nullptr;
  cudaStreamCaptureStatus cs{};
  const cudaGraphNode_t *deps = nullptr;
  size_t ndeps = 0;
  CondArgs ca{};
  ca.n = ss.n;
  if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg);
  for (int i = 0; i < ss.n && e == cudaSuccess; ++i) {
    ca.shape[i] = ss.k[i];
    e = cudaGraphConditionalHandleCreate(&ca.h[i], cg, 0, cudaGraphCondAssignDefault);
  }
  if (e == cudaSuccess) {
    k_graph_setcond<<<1, 1, 0, st>>>(ca, &d_ps->sum, g->d_gd);
    e = cudaGetLastError();
  }
  std::vector<cudaGraphNode_t> fork, join;
  if (e == cudaSuccess) e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &cg, &deps, nullptr, &ndeps);
  if (e == cudaSuccess) fork.assign(deps, deps + ndeps);
  FullArgs fa{};
  fa.b = none;
  fa.sp = sp;
  fa.order = d_order;
  fa.n_order = 0;
  fa.out = nullptr;
  fa.fwd = d_fwd;
  fa.tb = d_tb;
  fa.tbl = d_tbl;
  fa.strip_stride = strip_stride;
  fa.gd = g->d_gd;
  fa.gsum = &d_ps->sum;
  for (int i = 0; i < ss.n && e == cudaSuccess; ++i) {
    const int k = ss.k[i];
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = ca.h[i];
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddNode(&node, cg, fork.data(), nullptr, fork.size(), &np);
    if (e != cudaSuccess) break;
    join.push_back(node);
    e = cudaStreamBeginCaptureToGraph(st2, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                      cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) break;
    fa.counter = d_counters + k;
    fa.gshape = k;
    fa.strip_buf = d_strip[i];
    e = costs[k].packed ? launch_pack(fa, costs[k].R, ss.grid[i], st2)
                        : launch_full(fa, costs[k].R, ss.grid[i], st2);
    cudaGraph_t body = nullptr;
    const cudaError_t eb = cudaStreamEndCapture(st2, &body);
    if (e == cudaSuccess) e = eb;
  }
  if (e == cudaSuccess && !join.empty())
    e = cudaStreamUpdateCaptureDependencies(st, join.data(), nullptr, join.size(),
                                            cudaStreamSetCaptureDependencies);
  if (e == cudaSuccess)
    e = launch_trivial(none, sp, d_order, NP, nullptr, d_fwd, st, g->d_gd, &d_ps->sum);
  if (sp.traceback && e == cudaSuccess) {
    WalkArgs wa{};
    wa.b = none;
    wa.sp = sp;
    wa.order = d_order;
    wa.n_order = NP;
    wa.out = nullptr;
    wa.fwd = d_fwd;
    wa.tb = d_tb;
    wa.tbl = d_tbl;
    wa.stage = d_stage;
    wa.stage_off = d_stage_off;
    wa.gd = g->d_gd;
    e = launch_walk(wa, st);
    if (e == cudaSuccess) e = launch_scan_offsets(nullptr, NP, d_offs, d_total, st, g->d_gd);
    if (e == cudaSuccess) e = launch_compact(wa, NP, d_offs, nullptr, 0, nullptr, st);
  }
  if (e == cudaSuccess) {
    k_graph_finish<<<1, 1, 0, st>>>(g->d_gd, d_total, sp.traceback, g->d_status);
    e = cudaGetLastError();
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(st, &graph);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return e;
  }
  g->graph = graph;
  return cudaSuccess;
}

}  // namespace

extern "C" {

filtr_status filtr_graph_create(filtr_ctx *ctx, const filtr_params *params, uint32_t max_pairs,
                                uint32_t max_len, size_t workspace_bytes, filtr_graph **out) {
  if (!out) {
    set_error("filtr_graph_create: out is NULL");
    return FILTR_ERR_INVALID;
  }
  *out = nullptr;
  ScoreParams sp;
  filtr_status rc = to_score_params(params, &sp);
  if (rc != FILTR_OK) return rc;
  if (!ctx) {
    set_error("filtr_graph_create: ctx is NULL");
    return FILTR_ERR_INVALID;
  }
  if (sp.use_xdrop) {
    set_error("filtr_graph_create: X-drop / Z-drop batches rerun pairs by host decision; use "
              "filtr_align_batch");
    return FILTR_ERR_UNSUPPORTED;
  }
  if (max_pairs == 0 || max_len == 0 || max_len >= (1u << 30)) {
    set_error("filtr_graph_create: need 0 < max_pairs and 0 < max_len < 2^30");
    return FILTR_ERR_INVALID;
  }
  if (!score_range_ok(sp, max_len, max_len)) {
    set_error("filtr_graph_create: scores could exceed 2^28 (2^26 local) for max_len %u", max_len);
    return FILTR_ERR_UNSUPPORTED;
  }
  Ctx *c = reinterpret_cast<Ctx *>(ctx);
  cudaError_t e = cudaSetDevice(c->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  const ShapeCost *costs = c->tuned_costs(sp);
  if (!costs) costs = kDefaultShapeCost;

  // layout: fixed parts (capacity-sized), strip buffers per shape, staging,
  // traceback
  const ShapeSet ss = graph_shapes(c, sp, costs, max_len);
  const uint64_t stage_cap = sp.traceback ? (uint64_t)max_pairs * (2ull * max_len + 1) : 0;
  GCarve probe{nullptr};  // the same sequence of parts as capture() carves
  {
    probe.take<GraphDesc>(1);
    probe.take<DevPlanState>(1);
    probe.take<uint32_t>(max_pairs);
    probe.take<TbLayout>(max_pairs);
    probe.take<uint64_t>(max_pairs);
    probe.take<FwdOut>(max_pairs);
    probe.take<uint64_t>(max_pairs);
    probe.take<uint32_t>(64);
    probe.take<uint64_t>(4);
    probe.take<uint16_t>(max_pairs);
    probe.take<uint64_t>(max_pairs);
    probe.take<uint64_t>((max_pairs + DEV_PLAN_BLOCK - 1) / DEV_PLAN_BLOCK);
    for (int i = 0; i < ss.n; ++i) probe.take<int2>((size_t)ss.grid[i] * FULL_WARPS * (max_len + 2));
    if (sp.traceback) probe.take<uint32_t>(stage_cap);
    probe.take<uint32_t>(0);
  }
  const size_t fixed = probe.used;
  if (workspace_bytes < fixed + (sp.traceback ? 4096 : 0)) {
    set_error("filtr_graph_create: %zu bytes of workspace, the bounds need %zu before traceback",
              workspace_bytes, fixed);
    return FILTR_ERR_NOMEM;
  }
  const uint64_t tb_words = sp.traceback ? (workspace_bytes - fixed) / 4 : 0;

  Graph *g = new Graph;
  g->ctx = c;
  g->sp = sp;
  g->max_pairs = max_pairs;
  g->max_len = max_len;
  e = cudaMalloc(&g->mem, fixed + (size_t)tb_words * 4 + 256);
  if (e != cudaSuccess) {
    graph_free(g);
    return cuda_fail(e, "filtr_graph_create: device memory");
  }
  e = cudaHostAlloc(&g->h_status, 64, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&g->d_status, g->h_status, 0);
  if (e != cudaSuccess) {
    graph_free(g);
    return cuda_fail(e, "filtr_graph_create: status word");
  }
  *g->h_status = FILTR_OK;
  GCarve lay{g->mem};
  g->d_gd = lay.take<GraphDesc>(1);
  cudaStream_t st = nullptr, st2 = nullptr;
  e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    if (st) cudaStreamDestroy(st);
    graph_free(g);
    return cuda_fail(e, "cudaStreamCreate");
  }
  e = capture(g, costs, ss, tb_words, stage_cap, lay, st, st2);
  cudaStreamDestroy(st);
  cudaStreamDestroy(st2);
  if (e != cudaSuccess) {
    graph_free(g);
    return cuda_fail(e, "filtr_graph_create: capture");
  }
  size_t nroot = 1;
  cudaGraphNode_t root = nullptr;
  e = cudaGraphGetRootNodes(g->graph, &root, &nroot);
  cudaGraphNodeType type{};
  if (e == cudaSuccess && nroot == 1) e = cudaGraphNodeGetType(root, &type);
  if (e == cudaSuccess && (nroot != 1 || type != cudaGraphNodeTypeKernel)) e = cudaErrorUnknown;
  if (e == cudaSuccess) e = cudaGraphKernelNodeGetParams(root, &g->desc_params);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) {
    graph_free(g);
    return cuda_fail(e, "filtr_graph_create: instantiate");
  }
  g->desc_node = root;
  *out = reinterpret_cast<filtr_graph *>(g);
  return FILTR_OK;
}

filtr_status filtr_graph_launch(filtr_graph *graph, uint32_t n_pairs, const uint8_t *q_seq,
                                const uint64_t *q_off, const uint32_t *q_len, const uint8_t *r_seq,
                                const uint64_t *r_off, const uint32_t *r_len, filtr_result *out,
                                uint32_t *cigar, uint64_t cigar_cap, void *stream) {
  Graph *g = reinterpret_cast<Graph *>(graph);
  if (!g) {
    set_error("filtr_graph_launch: graph is NULL");
    return FILTR_ERR_INVALID;
  }
  if (n_pairs > g->max_pairs) {
    set_error("filtr_graph_launch: %u pairs, the graph holds %u", n_pairs, g->max_pairs);
    return FILTR_ERR_INVALID;
  }
  if (n_pairs == 0) return FILTR_OK;
  if (!q_seq || !q_off || !q_len || !r_seq || !r_off || !r_len || !out ||
      (g->sp.traceback && cigar_cap > 0 && !cigar)) {
    set_error("filtr_graph_launch: a batch pointer is NULL");
    return FILTR_ERR_INVALID;
  }
  GraphDesc d{};
  d.b = BatchDev{q_seq, r_seq, q_off, r_off, q_len, r_len};
  d.out = out;
  d.cigar = cigar;
  d.cap = cigar_cap;
  d.n = n_pairs;
  cudaKernelNodeParams kp = g->desc_params;
  void *args[2] = {&d, &g->d_gd};
  kp.kernelParams = args;
  kp.extra = nullptr;
  cudaError_t e = cudaSetDevice(g->ctx->device);
  if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(g->exec, g->desc_node, &kp);
  if (e == cudaSuccess) e = cudaGraphLaunch(g->exec, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "filtr_graph_launch");
  return FILTR_OK;
}

filtr_status filtr_graph_status(filtr_graph *graph) {
  Graph *g = reinterpret_cast<Graph *>(graph);
  if (!g) {
    set_error("filtr_graph_status: graph is NULL");
    return FILTR_ERR_INVALID;
  }
  const int32_t code = *reinterpret_cast<volatile int32_t *>(g->h_status);
  if (code == FILTR_ERR_INVALID)
    set_error("filtr_graph: a residue code >= the alphabet size or a sequence longer than max_len");
  else if (code == FILTR_ERR_NOMEM)
    set_error("filtr_graph: the batch's traceback exceeds the graph's workspace");
  else if (code == FILTR_ERR_CIGAR_CAP)
    set_error("filtr_graph: the CIGARs exceed cigar_cap");
  else if (code == FILTR_ERR_UNSUPPORTED)
    set_error("filtr_graph: the plan chose a tile shape the graph does not launch");
  return (filtr_status)code;
}

filtr_status filtr_graph_destroy(filtr_graph *graph) {
  Graph *g = reinterpret_cast<Graph *>(graph);
  if (!g) return FILTR_OK;
  cudaSetDevice(g->ctx->device);
  cudaDeviceSynchronize();
  graph_free(g);
  return FILTR_OK;
}

}  // extern "C"
