// Batched solves (include/accfem.h, accfem_batch_*): many handles advanced together, one persistent
// launch per Newton phase.  The paper solves one robot at a time; every member of a batch runs the
// block bodies of the single-instance kernels on its own buffers, so its iterates are those of
// accfem_solve.  Solves start and finish independently (continuous batching): accfem_batch_begin
// stages a solve, accfem_batch_advance starts the staged solves and runs a bounded number of
// iterations of everything in flight inside one CUDA graph (a conditional WHILE node whose body
// ends with the plan kernel), and finished members are collected with one gather and one copy.
#include <cstdio>
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/accfem.h"
#include "batch_host.h"

namespace accfem {
__global__ void element_batch_w2(const Inst* __restrict__ tab, const Plan* __restrict__ plan);
__global__ void element_batch_w4(const Inst* __restrict__ tab, const Plan* __restrict__ plan);
__global__ void element_batch_w8(const Inst* __restrict__ tab, const Plan* __restrict__ plan);
__global__ void collide_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan);
__global__ void collide_segment_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan);
__global__ void compact_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan);
__global__ void assemble_rhs_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan);
__global__ void bcr_level_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan, int j);
__global__ void bcr_bwd_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan, int j);
__global__ void contact_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan);
__global__ void step_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan);
__global__ void apply_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan);
__global__ void batch_begin_kernel(const Inst* __restrict__ tab, const Ctl* __restrict__ staged,
                                   const BatchBegin* __restrict__ bg);
__global__ void start_batch(const Inst* __restrict__ tab, const BatchBegin* __restrict__ bg);
__global__ void batch_plan_kernel(const Inst* __restrict__ tab, Plan* plan, int n_inst, int do_ctl, int max_passes,
                                  cudaGraphConditionalHandle h, int set_cond);

// Result gather: block j packs member members[j] at out + off[j]: 7 N poses (x, y, z, qw, qx, qy,
// qz, each N long), 6 base reaction values, then m rows of 9 values (free-node index, triangle,
// point 3, normal 3, force).
__global__ void __launch_bounds__(256) batch_pack_kernel(const Inst* __restrict__ tab, const int* __restrict__ members,
                                                         const long long* __restrict__ off, double* out) {
  const int mb = members[blockIdx.x];
  const Params& p = tab[mb].p;
  const Dev& d = tab[mb].d;
  const Ctl* c = d.ctl;
  double* o = out + off[blockIdx.x];
  const int N = p.N;
  const double* src[7] = {d.px, d.py, d.pz, d.qw, d.qx, d.qy, d.qz};
  for (int i = threadIdx.x; i < N; i += blockDim.x)
#pragma unroll
    for (int a = 0; a < 7; ++a) o[(size_t)a * N + i] = src[a][i];
  o += (size_t)7 * N;
  const bool iterated = c->nf > 0 && c->iter > 0;
  if (threadIdx.x < 6) o[threadIdx.x] = iterated ? d.elem[(size_t)c->k * kElemStride + 78 + threadIdx.x] : 0.0;
  o += 6;
  const int m = iterated ? c->m : 0;
  for (int r = threadIdx.x; r < m; r += blockDim.x) {
    double* q = o + 9 * (size_t)r;
    q[0] = (double)d.c_node[r];
    q[1] = (double)d.c_tri[r];
#pragma unroll
    for (int a = 0; a < 3; ++a) { q[2 + a] = d.c_pt[3 * r + a]; q[5 + a] = d.c_n[3 * r + a]; }
    q[8] = d.y[r];
  }
}
}  // namespace accfem

using namespace accfem;

namespace {

// Persistent grid of a batched phase kernel: resident blocks on every SM, at most the largest
// number of units the members can produce.
template <class K>
int persistent_grid(K kernel, int threads, long long max_units) {
  int dev = 0, sms = 0, occ = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, threads, 0);
  long long g = (long long)std::max(sms, 1) * std::max(occ, 1);
  g = std::min(g, std::max(max_units, 1ll));
  return (int)g;
}

// Element mapping of variant v: blocks of 2, 4 or 8 warps (one warp per element).
inline int variant_elem_w(int v) { return 2 << (v / 4); }
inline int variant_grid_shift(int v) { return v % 4; }

// The batched element phase with w warps per block.
void launch_element_batch(int w, bool pdl, dim3 grid, cudaStream_t st, const Inst* tab, const Plan* plan) {
  if (w == 8) launch_k(pdl, element_batch_w8, grid, dim3(256), st, tab, plan);
  else if (w == 4) launch_k(pdl, element_batch_w4, grid, dim3(128), st, tab, plan);
  else launch_k(pdl, element_batch_w2, grid, dim3(64), st, tab, plan);
}

// Enqueues one Newton iteration of every instance in flight on st (the body of the batch graph);
// returns the number of kernels.
int enqueue_batch_iteration(accfem_batch* b, cudaStream_t st, cudaGraphConditionalHandle cond, int set_cond) {
  const Inst* tab = b->d_tab;
  Plan* plan = b->d_plan;
  const int* g = b->grid;
  int n = 0;
  // the element phase and the collision + compaction phases both only read the poses: two branches
  cudaEventRecord(b->fork, st);
  cudaStreamWaitEvent(b->side, b->fork, 0);
  const bool pdl = b->pdl;
  launch_element_batch(b->elem_w, pdl, dim3(g[PH_ELEM]), b->side, tab, plan); ++n;
  cudaEventRecord(b->join, b->side);
  launch_k(pdl, collide_batch, dim3(g[PH_COLL]), dim3(128), st, tab, plan); ++n;
  if (b->has_segment) { launch_k(pdl, collide_segment_batch, dim3(g[PH_COLL]), dim3(128), st, tab, plan); ++n; }
  launch_k(pdl, compact_batch, dim3(g[PH_COMPACT]), dim3(1024), st, tab, plan); ++n;
  cudaStreamWaitEvent(st, b->join, 0);
  launch_k(pdl, assemble_rhs_batch, dim3(g[PH_ASM]), dim3(32, 6), st, tab, plan); ++n;
  for (int j = 0; j < b->levels; ++j) { launch_k(pdl, bcr_level_batch, dim3(g[PH_LEV0 + j]), dim3(192), st, tab, plan, j); ++n; }
  for (int j = b->levels - 1; j >= 0; --j) { launch_k(pdl, bcr_bwd_batch, dim3(g[PH_BWD0 + j]), dim3(96), st, tab, plan, j); ++n; }
  launch_ks(pdl, contact_batch, dim3(g[PH_CONTACT]), dim3(256), b->has_admm ? kAdmmSmemBytes : kBatchWSmemBytes, st, tab, plan); ++n;
  launch_k(pdl, step_batch, dim3(g[PH_STEP]), dim3(32, 6), st, tab, plan); ++n;
  launch_k(pdl, apply_batch, dim3(g[PH_APPLY]), dim3(128), st, tab, plan); ++n;
  launch_k(pdl, batch_plan_kernel, dim3(1), dim3(1024), st, tab, plan, b->n, 1, 0, cond, set_cond); ++n;
  return n;
}

// Persistent grids of the phase kernels at the full resident size (units: the largest number of
// units the members can produce).
void full_grids(accfem_batch* b, int elem_w, int* grid) {
  long long units[kPhases] = {};
  for (accfem_handle* h : b->members)
    for (int ph = 0; ph < kPhases; ++ph) units[ph] += (long long)phase_gx(ph, h->p.M) * phase_gy(ph);
  for (int ph = 0; ph < kPhases; ++ph) grid[ph] = 1;
  const long long eu = (units[PH_ELEM] * kWarpsPerElemBlock + elem_w - 1) / elem_w;   // blocks of elem_w warps
  grid[PH_ELEM] = elem_w == 8 ? persistent_grid(element_batch_w8, 256, eu)
                : elem_w == 4 ? persistent_grid(element_batch_w4, 128, eu)
                              : persistent_grid(element_batch_w2, 64, eu);
  grid[PH_COLL] = persistent_grid(collide_batch, 128, units[PH_COLL]);
  grid[PH_COMPACT] = persistent_grid(compact_batch, 1024, units[PH_COMPACT]);
  grid[PH_ASM] = persistent_grid(assemble_rhs_batch, 192, units[PH_ASM]);
  grid[PH_CONTACT] = persistent_grid(contact_batch, 256, units[PH_CONTACT]);
  grid[PH_STEP] = persistent_grid(step_batch, 192, units[PH_STEP]);
  grid[PH_APPLY] = persistent_grid(apply_batch, 128, units[PH_APPLY]);
  for (int j = 0; j < b->levels; ++j) {
    grid[PH_LEV0 + j] = persistent_grid(bcr_level_batch, 192, units[PH_LEV0 + j]);
    grid[PH_BWD0 + j] = persistent_grid(bcr_bwd_batch, 96, units[PH_BWD0 + j]);
  }
}

// Graph of variant v: every persistent grid divided by 2^(v % 4) (at least one block), element blocks
// of 2 << (v / 4) warps.
bool build_graph(accfem_batch* b, int v) {
  accfem_batch::Variant& g = b->variants[v];
  if (g.exec) return true;
  int full[kPhases];
  b->elem_w = variant_elem_w(v);
  full_grids(b, b->elem_w, full);
  for (int ph = 0; ph < kPhases; ++ph) b->grid[ph] = std::max(1, full[ph] >> variant_grid_shift(v));
  cudaGraphConditionalHandle cond;
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t node;
  if (!bok(b, cudaGraphCreate(&g.graph, 0), "cudaGraphCreate") ||
      !bok(b, cudaGraphConditionalHandleCreate(&cond, g.graph, 1, cudaGraphCondAssignDefault), "conditional handle"))
    return false;
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if (!bok(b, cudaGraphAddNode(&node, g.graph, nullptr, nullptr, 0, &cp), "conditional node")) return false;
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  cudaStream_t st = b->stream;
  if (!bok(b, cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed), "begin capture"))
    return false;
  b->body_kernels = enqueue_batch_iteration(b, st, cond, 1);
  cudaError_t ce = cudaStreamEndCapture(st, &body);
  if (!bok(b, ce, "end capture") || !bok(b, cudaGraphInstantiate(&g.exec, g.graph, 0), "instantiate graph")) {
    cudaGetLastError();
    cudaGraphDestroy(g.graph);
    g.graph = nullptr;
    g.exec = nullptr;
    if (b->pdl) {                 // programmatic edges refused inside the loop body: capture without them
      std::fprintf(stderr, "accfem: programmatic dependent launch refused in the batch graph; plain launches\n");
      b->pdl = false;
      return build_graph(b, v);
    }
    return false;
  }
  for (int ph = 0; ph < kPhases; ++ph) g.grid[ph] = b->grid[ph];
  return true;
}

template <typename T>
bool balloc(accfem_batch* b, T** dptr, size_t count) {
  if (count == 0) count = 1;
  if (cudaMalloc((void**)dptr, count * sizeof(T)) != cudaSuccess) {
    b->err = "cudaMalloc failed";
    return false;
  }
  cudaMemset(*dptr, 0, count * sizeof(T));
  b->dev_bytes += (int64_t)(count * sizeof(T));
  return true;
}

template <typename T>
bool bhost(accfem_batch* b, T** hptr, size_t count) {
  if (count == 0) count = 1;
  if (cudaMallocHost((void**)hptr, count * sizeof(T)) != cudaSuccess) {
    b->err = "cudaMallocHost failed";
    return false;
  }
  std::memset(*hptr, 0, count * sizeof(T));
  return true;
}

}  // namespace

extern "C" {

void accfem_batch_destroy(accfem_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& g : b->variants) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    if (g.graph) cudaGraphDestroy(g.graph);
  }
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  for (void* p : {(void*)b->d_tab, (void*)b->d_plan, (void*)b->d_ctl, (void*)b->d_stage, (void*)b->d_begin,
                  (void*)b->d_members, (void*)b->d_off, (void*)b->d_pack, (void*)b->d_tips})
    if (p) cudaFree(p);
  for (void* p : {(void*)b->h_ctl, (void*)b->h_stage, (void*)b->h_begin, (void*)b->h_members, (void*)b->h_off,
                  (void*)b->h_pack, (void*)b->h_passes, (void*)b->h_tips})
    if (p) cudaFreeHost(p);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->join) cudaEventDestroy(b->join);
  if (b->side) cudaStreamDestroy(b->side);
  if (b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

accfem_status accfem_batch_create(accfem_handle* const* members, int32_t n_members, accfem_batch** out) {
  if (!out) return ACCFEM_E_INVALID_ARG;
  *out = nullptr;
  if (!members || n_members < 1 || n_members > kMaxBatch) return ACCFEM_E_INVALID_ARG;
  for (int i = 0; i < n_members; ++i) {
    if (!members[i]) return ACCFEM_E_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (members[j] == members[i]) return ACCFEM_E_INVALID_ARG;
    // every member on the current device: the batch's kernels read all members' buffers
    if (!accfem_on_device(members[i], "accfem_batch_create")) return ACCFEM_E_INVALID_ARG;
    if (members[i]->p.lcp_mode == kLcpPrimalAdmm) return ACCFEM_E_INVALID_ARG;   // single-instance solver only
  }
  accfem_batch* b = new accfem_batch();
  b->members.assign(members, members + n_members);
  b->n = n_members;
  b->state.assign(n_members, 0);
  b->solved.assign(n_members, 0);
  size_t pack = 0;
  int max_m = 0;
  for (accfem_handle* h : b->members) {
    b->max_nodes = std::max(b->max_nodes, h->p.N);
    b->has_segment = b->has_segment || h->p.contact_model == kContactSegment;
    b->has_admm = b->has_admm || h->p.lcp_mode == kLcpAdmm;
    max_m = std::max(max_m, h->p.M);
    pack += (size_t)7 * h->p.N + 6 + (size_t)9 * h->p.m_cap;
  }
  while (b->levels < kMaxLevels && phase_gx(PH_LEV0 + b->levels, max_m) > 0) ++b->levels;
  b->pack_cap = pack;
  {
    const char* lm = std::getenv("ACCFEM_LAUNCH");
    b->stream_mode = lm && std::strcmp(lm, "stream") == 0;
    b->pdl = pdl_default();
  }
  bool ok = bok(b, cudaFuncSetAttribute(contact_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdmmSmemBytes),
                "contact kernel shared memory") &&
            bok(b, cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "cudaStreamCreate") &&
            bok(b, cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking), "cudaStreamCreate") &&
            bok(b, cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming), "cudaEventCreate") &&
            bok(b, cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming), "cudaEventCreate") &&
            balloc(b, &b->d_tab, b->n) && balloc(b, &b->d_plan, 1) && balloc(b, &b->d_ctl, b->n) &&
            balloc(b, &b->d_stage, b->n) && balloc(b, &b->d_begin, b->n) && balloc(b, &b->d_members, b->n) &&
            balloc(b, &b->d_off, b->n) && balloc(b, &b->d_pack, pack) && balloc(b, &b->d_tips, (size_t)8 * b->n) &&
            bhost(b, &b->h_tips, (size_t)8 * b->n) && bhost(b, &b->h_ctl, b->n) &&
            bhost(b, &b->h_stage, b->n) && bhost(b, &b->h_begin, b->n) && bhost(b, &b->h_members, b->n) &&
            bhost(b, &b->h_off, b->n) && bhost(b, &b->h_pack, pack) && bhost(b, &b->h_passes, 4);
  if (!ok) {
    accfem_batch_destroy(b);
    return ACCFEM_E_NOMEM;
  }
  std::vector<Inst> tab(b->n);
  for (int i = 0; i < b->n; ++i) {
    tab[i].p = b->members[i]->p;
    tab[i].d = b->members[i]->d;
    tab[i].d.ctl = b->d_ctl + i;
  }
  if (!bok(b, cudaMemcpy(b->d_tab, tab.data(), sizeof(Inst) * b->n, cudaMemcpyHostToDevice), "upload batch table") ||
      !bok(b, cudaEventCreate(&b->ev0), "event") || !bok(b, cudaEventCreate(&b->ev1), "event") ||
      !build_graph(b, 0)) {
    accfem_batch_destroy(b);
    return ACCFEM_E_CUDA;
  }
  *out = b;
  return ACCFEM_OK;
}

accfem_status accfem_batch_set_stream(accfem_batch* b, void* stream) {
  if (!b) return ACCFEM_E_INVALID_ARG;
  b->user_stream = (cudaStream_t)stream;
  return ACCFEM_OK;
}

accfem_status accfem_batch_begin(accfem_batch* b, int32_t member, const double* cable_tensions, double insertion) {
  if (!b) return ACCFEM_E_INVALID_ARG;
  if (member < 0 || member >= b->n) return bfail(b, ACCFEM_E_INVALID_ARG, "member index out of range");
  if (b->state[member] != 0) return bfail(b, ACCFEM_E_INVALID_ARG, "member has a solve staged or in flight");
  accfem_handle* h = b->members[member];
  const Params& p = h->p;
  if (!(insertion >= 0.0 && insertion <= p.L)) return bfail(b, ACCFEM_E_INVALID_ARG, "insertion outside [0, length]");
  if (p.n_cables > 0 && !cable_tensions) return bfail(b, ACCFEM_E_INVALID_ARG, "NULL cable tensions");
  for (int j = 0; j < p.n_cables; ++j)
    if (!(cable_tensions[j] >= 0.0) || !std::isfinite(cable_tensions[j]))
      return bfail(b, ACCFEM_E_INVALID_ARG, "cable tensions must be finite and non-negative");
  const int k = std::min(std::max(accfem_last_prescribed(p.L, p.M, insertion), 0), p.M);
  Ctl& c = b->h_stage[b->n_begin];
  std::memset(&c, 0, sizeof(Ctl));
  c.k = k;
  c.nf = p.M - k;
  c.m_prev = -1;
  c.rho = p.beta0;
  c.load_mode = 0;
  c.delta = insertion;
  c.live = c.nf > 0 ? 1 : 0;
  c.frame = h->frame_iters > 0 ? 1 : 0;
  for (int j = 0; j < p.n_cables; ++j) c.tension[j] = cable_tensions[j];
  BatchBegin& g = b->h_begin[b->n_begin];
  g.member = member;
  g.mode = h->has_state ? 1 : 0;
  g.k = k;
  g.pad = 0;
  g.delta = insertion;
  g.delta_old = h->delta;
  ++b->n_begin;
  h->has_state = true;
  h->delta = insertion;
  b->state[member] = 1;
  return ACCFEM_OK;
}

accfem_status accfem_batch_advance(accfem_batch* b, int32_t max_iters, int32_t* n_in_flight) {
  if (!b || max_iters < 1) return bfail(b, ACCFEM_E_INVALID_ARG, "NULL batch or max_iters < 1");
  b->err.clear();
  if (!accfem_on_device(b->members[0], "accfem_batch_advance"))
    return bfail(b, ACCFEM_E_INVALID_ARG, b->members[0]->err);
  cudaStream_t st = b->work();
  if (b->n_begin > 0) {
    const int nb = b->n_begin;
    if (!bok(b, cudaMemcpyAsync(b->d_stage, b->h_stage, sizeof(Ctl) * nb, cudaMemcpyHostToDevice, st), "upload control") ||
        !bok(b, cudaMemcpyAsync(b->d_begin, b->h_begin, sizeof(BatchBegin) * nb, cudaMemcpyHostToDevice, st), "upload begin"))
      return ACCFEM_E_CUDA;
    b->h2d += (sizeof(Ctl) + sizeof(BatchBegin)) * nb;
    const dim3 grid((b->max_nodes + 127) / 128, nb);
    batch_begin_kernel<<<grid, 128, 0, st>>>(b->d_tab, b->d_stage, b->d_begin);
    start_batch<<<grid, 128, 0, st>>>(b->d_tab, b->d_begin);
    b->launches += 2;
    for (int i = 0; i < nb; ++i) b->state[b->h_begin[i].member] = 2;
    b->n_begin = 0;
  }
  int flying = 0;
  int tuned_variant = -1;
  for (int i = 0; i < b->n; ++i) flying += b->state[i] == 2;
  if (flying > 0) {
    batch_plan_kernel<<<1, 1024, 0, st>>>(b->d_tab, b->d_plan, b->n, 0, max_iters, cudaGraphConditionalHandle(), 0);
    ++b->launches;
    if (!bok(b, cudaGetLastError(), "kernel launch")) return ACCFEM_E_CUDA;
    int v = b->variant;
    if (b->tune_left > 0) {                 // autotuning: the variants take turns, one advance each
      v = b->tune_next;
      b->tune_next = (b->tune_next + 1) % accfem_batch::kVariants;
      if (!build_graph(b, v)) return ACCFEM_E_CUDA;
    }
    for (int ph = 0; ph < kPhases; ++ph) b->grid[ph] = b->variants[v].grid[ph];
    b->elem_w = variant_elem_w(v);
    if (b->stream_mode) {
      // host-driven passes (kernels visible to profilers): stop when nothing iterates
      for (int pass = 0; pass < max_iters; ++pass) {
        b->launches += enqueue_batch_iteration(b, st, cudaGraphConditionalHandle(), 0);
        if (!bok(b, cudaMemcpyAsync(b->h_passes + 1, &b->d_plan->n_act, sizeof(int), cudaMemcpyDeviceToHost, st),
                 "read plan") ||
            !bok(b, cudaStreamSynchronize(st), "batch iteration"))
          return ACCFEM_E_CUDA;
        if (b->h_passes[1] == 0) break;
      }
    } else {
      const bool timed = b->tune_left > 0;
      if ((timed && !bok(b, cudaEventRecord(b->ev0, st), "event")) ||
          !bok(b, cudaGraphLaunch(b->variants[v].exec, st), "launch batch graph") ||
          (timed && !bok(b, cudaEventRecord(b->ev1, st), "event")))
        return ACCFEM_E_CUDA;
      tuned_variant = timed ? v : -1;
    }
  }
  if (!bok(b, cudaMemcpyAsync(b->h_ctl, b->d_ctl, sizeof(Ctl) * b->n, cudaMemcpyDeviceToHost, st), "read control") ||
      !bok(b, cudaMemcpyAsync(b->h_passes, &b->d_plan->passes, sizeof(int), cudaMemcpyDeviceToHost, st), "read plan") ||
      !bok(b, cudaStreamSynchronize(st), "batch advance"))
    return ACCFEM_E_CUDA;
  b->d2h += sizeof(Ctl) * b->n + sizeof(int);
  if (flying > 0 && !b->stream_mode) b->launches += (int64_t)b->body_kernels * std::max(*b->h_passes, 1);
  if (tuned_variant >= 0) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->ev0, b->ev1);
    b->tune_ms[tuned_variant] += ms;
    b->tune_passes[tuned_variant] += std::max(*b->h_passes, 1);
    if (--b->tune_left == 0) {               // keep the variant with the least time per pass
      int best = 0;
      for (int k = 1; k < accfem_batch::kVariants; ++k)
        if (b->tune_passes[k] > 0 &&
            b->tune_ms[k] / b->tune_passes[k] < b->tune_ms[best] / std::max<int64_t>(b->tune_passes[best], 1))
          best = k;
      b->variant = best;
    }
  }
  int left = 0;
  for (int i = 0; i < b->n; ++i) {
    if (b->state[i] != 2) {
      left += b->state[i] == 1;
      continue;
    }
    if (b->h_ctl[i].live) {
      ++left;
      continue;
    }
    b->state[i] = 0;
    b->solved[i] = 1;
    *b->members[i]->h_ctl = b->h_ctl[i];
  }
  if (n_in_flight) *n_in_flight = left;
  return ACCFEM_OK;
}

accfem_status accfem_batch_poll(const accfem_batch* b, int32_t member, int32_t* done, accfem_status* solve_status,
                                int32_t* newton_iters) {
  if (!b || member < 0 || member >= b->n || !done) return ACCFEM_E_INVALID_ARG;
  *done = b->state[member] == 0 ? 1 : 0;
  const Ctl& c = b->h_ctl[member];
  const bool have = *done && b->solved[member];
  if (solve_status) *solve_status = have ? outcome(c) : ACCFEM_OK;
  if (newton_iters) *newton_iters = have ? c.iter : 0;
  return ACCFEM_OK;
}

accfem_status accfem_batch_results(accfem_batch* b, const int32_t* members, int32_t count, accfem_result* out,
                                   accfem_status* statuses) {
  if (b) b->err.clear();
  if (!b || count < 0 || count > b->n || (count > 0 && (!members || !out))) return bfail(b, ACCFEM_E_INVALID_ARG, "bad arguments");
  if (count == 0) return ACCFEM_OK;
  long long off = 0;
  std::vector<int> ms(count);
  for (int j = 0; j < count; ++j) {
    const int i = members[j];
    if (i < 0 || i >= b->n || b->state[i] != 0 || !b->solved[i])
      return bfail(b, ACCFEM_E_INVALID_ARG, "member has no finished solve");
    const Ctl& c = b->h_ctl[i];
    const int m = (c.nf > 0 && c.iter > 0) ? c.m : 0;
    b->h_members[j] = i;
    b->h_off[j] = off;
    ms[j] = m;
    off += (long long)7 * b->members[i]->p.N + 6 + 9ll * m;
  }
  if ((size_t)off > b->pack_cap) return bfail(b, ACCFEM_E_INVALID_ARG, "result larger than the gather buffer");
  cudaStream_t st = b->work();
  if (!bok(b, cudaMemcpyAsync(b->d_members, b->h_members, sizeof(int) * count, cudaMemcpyHostToDevice, st), "upload list") ||
      !bok(b, cudaMemcpyAsync(b->d_off, b->h_off, sizeof(long long) * count, cudaMemcpyHostToDevice, st), "upload offsets"))
    return ACCFEM_E_CUDA;
  batch_pack_kernel<<<count, 256, 0, st>>>(b->d_tab, b->d_members, b->d_off, b->d_pack);
  ++b->launches;
  if (!bok(b, cudaGetLastError(), "gather results") ||
      !bok(b, cudaMemcpyAsync(b->h_pack, b->d_pack, sizeof(double) * off, cudaMemcpyDeviceToHost, st), "download results") ||
      !bok(b, cudaStreamSynchronize(st), "download results"))
    return ACCFEM_E_CUDA;
  b->h2d += (sizeof(int) + sizeof(long long)) * count;
  b->d2h += sizeof(double) * off;
  accfem_status first = ACCFEM_OK;
  for (int j = 0; j < count; ++j) {
    const int i = members[j];
    const Ctl& c = b->h_ctl[i];
    const int N = b->members[i]->p.N, m = ms[j];
    const double* s = b->h_pack + b->h_off[j];
    accfem_result& r = out[j];
    accfem_status st_j = outcome(c);
    if (r.node_pos)
      for (int n = 0; n < N; ++n)
        for (int a = 0; a < 3; ++a) r.node_pos[3 * n + a] = s[(size_t)a * N + n];
    if (r.node_quat)
      for (int n = 0; n < N; ++n)
        for (int a = 0; a < 4; ++a) r.node_quat[4 * n + a] = s[(size_t)(3 + a) * N + n];
    s += (size_t)7 * N;
    for (int a = 0; a < 6; ++a) r.base_reaction[a] = s[a];
    s += 6;
    r.newton_iters = c.iter;
    r.contact_iters = c.lcp_pivots;
    r.residual = c.nf > 0 ? __builtin_bit_cast(double, (unsigned long long)c.res_bits) : 0.0;
    r.n_contacts = m;
    const int nw = std::min(m, std::max(r.contact_capacity, 0));
    for (int q = 0; q < nw; ++q) {
      const double* row = s + 9 * (size_t)q;
      if (r.contact_node) r.contact_node[q] = c.k + 1 + (int)row[0];
      if (r.contact_tri) r.contact_tri[q] = (int)row[1];
      for (int a = 0; a < 3; ++a) {
        if (r.contact_point) r.contact_point[3 * q + a] = row[2 + a];
        if (r.contact_normal) r.contact_normal[3 * q + a] = row[5 + a];
      }
      if (r.contact_force) r.contact_force[q] = row[8];
    }
    if (m > r.contact_capacity && st_j == ACCFEM_OK) st_j = ACCFEM_E_CONTACT_CAPACITY;
    if (statuses) statuses[j] = st_j;
    if (first == ACCFEM_OK && st_j != ACCFEM_OK) {
      first = st_j;
      b->err = "member " + std::to_string(i) + ": " + accfem_solve_message(c, st_j);
    }
  }
  return first;
}

accfem_status accfem_batch_solve(accfem_batch* b, const double* cable_tensions, const double* insertions,
                                 const int32_t* mask, accfem_status* statuses, accfem_result* results) {
  if (!b || !insertions) return bfail(b, ACCFEM_E_INVALID_ARG, "NULL argument");
  std::vector<int32_t> list;
  for (int i = 0; i < b->n; ++i) {
    if (mask && !mask[i]) continue;
    if (b->state[i] != 0) return bfail(b, ACCFEM_E_INVALID_ARG, "member has a solve staged or in flight");
    list.push_back(i);
  }
  for (int32_t i : list) {
    accfem_status s = accfem_batch_begin(b, i, cable_tensions ? cable_tensions + (size_t)ACCFEM_MAX_CABLES * i : nullptr,
                                         insertions[i]);
    if (s != ACCFEM_OK) return s;
  }
  int cap = 1;
  for (int32_t i : list) cap = std::max(cap, b->members[i]->max_newton);
  int32_t left = 0;
  accfem_status s = accfem_batch_advance(b, cap, &left);
  for (int guard = 0; s == ACCFEM_OK && left > 0 && guard < 4; ++guard) s = accfem_batch_advance(b, cap, &left);
  if (s != ACCFEM_OK) return s;
  if (left > 0) return bfail(b, ACCFEM_E_CUDA, "batch did not finish within its iteration caps");
  accfem_status first = ACCFEM_OK;
  if (results) {
    std::vector<accfem_result> tmp(list.size());
    std::vector<accfem_status> st(list.size());
    for (size_t j = 0; j < list.size(); ++j) tmp[j] = results[list[j]];
    accfem_status r = accfem_batch_results(b, list.data(), (int32_t)list.size(), tmp.data(), st.data());
    if (r == ACCFEM_E_CUDA || r == ACCFEM_E_INVALID_ARG) return r;
    first = r;
    for (size_t j = 0; j < list.size(); ++j) {
      results[list[j]] = tmp[j];
      if (statuses) statuses[list[j]] = st[j];
    }
  } else {
    for (int32_t i : list) {
      accfem_status o = outcome(b->h_ctl[i]);
      if (statuses) statuses[i] = o;
      if (first == ACCFEM_OK && o != ACCFEM_OK) first = o;
    }
  }
  return first;
}

accfem_status accfem_batch_time_phase(accfem_batch* b, accfem_kernel kernel, int32_t reps, double* us, int64_t* items) {
  if (!b || !us || reps < 1 || reps > 1000) return bfail(b, ACCFEM_E_INVALID_ARG, "NULL argument or reps outside 1..1000");
  if (kernel != ACCFEM_KERNEL_ELEMENT && kernel != ACCFEM_KERNEL_COLLIDE && kernel != ACCFEM_KERNEL_ASSEMBLE)
    return bfail(b, ACCFEM_E_INVALID_ARG, "only the element, collision and assembly phases can be timed");
  if (!accfem_on_device(b->members[0], "accfem_batch_time_phase"))
    return bfail(b, ACCFEM_E_INVALID_ARG, b->members[0]->err);
  cudaStream_t st = b->work();
  // the plan of the next iteration: members still iterating after the last advance
  int n_act = 0;
  if (!bok(b, cudaMemcpyAsync(&n_act, &b->d_plan->n_act, sizeof(int), cudaMemcpyDeviceToHost, st), "read plan") ||
      !bok(b, cudaStreamSynchronize(st), "read plan"))
    return ACCFEM_E_CUDA;
  if (n_act <= 0) return bfail(b, ACCFEM_E_INVALID_ARG, "no member is iterating (advance with solves in flight first)");
  std::vector<int> act(n_act);
  if (!bok(b, cudaMemcpy(act.data(), b->d_plan->act, sizeof(int) * n_act, cudaMemcpyDeviceToHost), "read plan"))
    return ACCFEM_E_CUDA;
  int64_t n_items = 0;
  for (int i : act) n_items += std::max(b->h_ctl[i].nf, 0);
  // a 256 MiB buffer written before every timed launch evicts the 129 MB L2
  const size_t flush_bytes = (size_t)256 << 20;
  void* flush = nullptr;
  if (!bok(b, cudaMalloc(&flush, flush_bytes), "flush buffer")) return ACCFEM_E_NOMEM;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int* g = b->variants[b->variant].grid;
  double total = 0.0;
  bool ok = true;
  for (int r = 0; r < reps && ok; ++r) {
    ok = bok(b, cudaMemsetAsync(flush, r & 0xff, flush_bytes, st), "flush L2");
    cudaEventRecord(e0, st);
    switch (kernel) {
      case ACCFEM_KERNEL_ELEMENT:
        launch_element_batch(variant_elem_w(b->variant), false, dim3(g[PH_ELEM]), st, b->d_tab, b->d_plan); break;
      case ACCFEM_KERNEL_COLLIDE: collide_batch<<<g[PH_COLL], 128, 0, st>>>(b->d_tab, b->d_plan); break;
      default: assemble_rhs_batch<<<g[PH_ASM], dim3(32, 6), 0, st>>>(b->d_tab, b->d_plan); break;
    }
    cudaEventRecord(e1, st);
    ++b->launches;
    float ms = 0.f;
    ok = ok && bok(b, cudaGetLastError(), "phase launch") && bok(b, cudaEventSynchronize(e1), "time phase");
    cudaEventElapsedTime(&ms, e0, e1);
    total += ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(flush);
  if (!ok) return ACCFEM_E_CUDA;
  *us = 1000.0 * total / reps;
  if (items) *items = n_items;
  return ACCFEM_OK;
}

accfem_status accfem_batch_autotune(accfem_batch* b, int32_t trials) {
  if (!b || trials < 1 || trials > 1000) return bfail(b, ACCFEM_E_INVALID_ARG, "trials must be in 1..1000");
  for (int k = 0; k < accfem_batch::kVariants; ++k) { b->tune_ms[k] = 0.0; b->tune_passes[k] = 0; }
  b->tune_left = trials * accfem_batch::kVariants;
  b->tune_next = 0;
  return ACCFEM_OK;
}

accfem_status accfem_batch_tuning(const accfem_batch* b, int32_t* variant, double* ms_per_pass) {
  if (!b || !variant) return ACCFEM_E_INVALID_ARG;
  *variant = b->tune_left > 0 ? -1 : b->variant;
  if (ms_per_pass)
    for (int k = 0; k < accfem_batch::kVariants; ++k)
      ms_per_pass[k] = b->tune_passes[k] > 0 ? b->tune_ms[k] / b->tune_passes[k] : -1.0;
  return ACCFEM_OK;
}

accfem_status accfem_batch_transfer_bytes(const accfem_batch* b, int64_t* h2d, int64_t* d2h) {
  if (!b || !h2d || !d2h) return ACCFEM_E_INVALID_ARG;
  *h2d = b->h2d;
  *d2h = b->d2h;
  return ACCFEM_OK;
}

int64_t accfem_batch_kernel_launches(const accfem_batch* b) { return b ? b->launches : 0; }

const char* accfem_batch_last_error(const accfem_batch* b) { return b ? b->err.c_str() : ""; }

}  // extern "C"
