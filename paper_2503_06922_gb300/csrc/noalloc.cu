// Collision query that allocates nothing (accfem_detect_contacts_noalloc in include/accfem.h).
//
// Same constraint rule and the same two-pass FP32 prefilter / exact FP64 test as collide_kernel,
// for node positions the caller passes, with the per-node row lists kept in one file-scope
// device array instead of memory owned by the handle.  Sized for at most kNoAllocMaxNodes nodes
// and kCpn rows per node, the solve's own per-node limit (about 4 MB); every GPU that loads the
// library holds this array until the process exits.
#include <cstring>

#include "../../include/accfem.h"
#include "common.cuh"
#include "collide_geom.cuh"

namespace accfem {

constexpr int kNoAllocMaxNodes = 4096;
constexpr int kNoAllocCpn = kCpn;     // rows per node in the fixed array, as in collide_kernel
static_assert(kNoAllocCpn == kCpn, "the query keeps the solve's per-node row limit");

struct NoAllocScratch {
  int ncon[kNoAllocMaxNodes];
  int tri[kNoAllocMaxNodes * kNoAllocCpn];
  double pt[kNoAllocMaxNodes * kNoAllocCpn * 3];
  double nrm[kNoAllocMaxNodes * kNoAllocCpn * 3];
  double gap[kNoAllocMaxNodes * kNoAllocCpn];
  int status;     // 0, or ST_CAPACITY when a node has too many candidates or rows
  int n_rows;     // rows of the last call
};

// The scratch of every call; in host code this name is only a stand-in (use the symbol address).
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// One warp per node: the rows of node i (position pos[3i..3i+2]) into the scratch lists.
__global__ void __launch_bounds__(128) detect_noalloc_kernel(Params p, Dev d, const double* pos, int n,
                                                             NoAllocScratch* sc) {
  __shared__ Surv s_surv[4][kSurvCap];
  __shared__ int s_ns[4];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int f = blockIdx.x * 4 + wib;
  if (f >= n) return;
  if (lane == 0) s_ns[wib] = 0;
  __syncwarp();
  const double pn[3] = {pos[3 * f], pos[3 * f + 1], pos[3 * f + 2]};
  const double thr = p.r_o + p.act;
  int lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = (int)floor((pn[a] - p.g_rq - p.g_org[a]) / p.g_h);
    hi[a] = (int)floor((pn[a] + p.g_rq - p.g_org[a]) / p.g_h);
    lo[a] = max(lo[a], 0);
    hi[a] = min(hi[a], p.g_dim[a] - 1);
  }
  const float thr32 = (float)(thr + p.eps_d);
  float dmin = 3.0e38f;
  for (int cz = lo[2]; cz <= hi[2]; ++cz)
    for (int cy = lo[1]; cy <= hi[1]; ++cy)
      for (int cx = lo[0]; cx <= hi[0]; ++cx) {
        int cell = (cz * p.g_dim[1] + cy) * p.g_dim[0] + cx;
        int s0 = d.cell_start[cell], s1 = d.cell_start[cell + 1];
        if (s0 == s1) continue;
        float pc[3] = {(float)(pn[0] - (p.g_org[0] + (cx + 0.5) * p.g_h)),
                       (float)(pn[1] - (p.g_org[1] + (cy + 0.5) * p.g_h)),
                       (float)(pn[2] - (p.g_org[2] + (cz + 0.5) * p.g_h))};
        for (int s = s0 + lane; s < s1; s += 32) {
          float va, vb, vc;
          dmin = fminf(dmin, sqrtf(tri_dist2_f32(pc, d.tri32 + (size_t)s * 9, va, vb, vc)));
        }
      }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
  const float dmin_keep = dmin + (float)(2.0 * p.eps_d);
  for (int cz = lo[2]; cz <= hi[2]; ++cz)
    for (int cy = lo[1]; cy <= hi[1]; ++cy)
      for (int cx = lo[0]; cx <= hi[0]; ++cx) {
        int cell = (cz * p.g_dim[1] + cy) * p.g_dim[0] + cx;
        int s0 = d.cell_start[cell], s1 = d.cell_start[cell + 1];
        if (s0 == s1) continue;
        float pc[3] = {(float)(pn[0] - (p.g_org[0] + (cx + 0.5) * p.g_h)),
                       (float)(pn[1] - (p.g_org[1] + (cy + 0.5) * p.g_h)),
                       (float)(pn[2] - (p.g_org[2] + (cz + 0.5) * p.g_h))};
        for (int s0l = s0; s0l < s1; s0l += 32) {
          int s = s0l + lane;
          bool keep = false;
          if (s < s1) {
            float va, vb, vc;
            float dd = sqrtf(tri_dist2_f32(pc, d.tri32 + (size_t)s * 9, va, vb, vc));
            float tol = -((float)kFaceBand + p.eps_b) * (va + vb + vc);
            bool near_in = (va >= tol) && (vb >= tol) && (vc >= tol);
            keep = (dd <= thr32) && (near_in || dd <= dmin_keep);
          }
          if (keep) {
            int t = d.cell_tri[s];
            const int* tv = d.T + 3 * (size_t)t;
            double A[3] = {d.V[3 * tv[0]], d.V[3 * tv[0] + 1], d.V[3 * tv[0] + 2]};
            double Bv[3] = {d.V[3 * tv[1]], d.V[3 * tv[1] + 1], d.V[3 * tv[1] + 2]};
            double Cv[3] = {d.V[3 * tv[2]], d.V[3 * tv[2] + 1], d.V[3 * tv[2] + 2]};
            Surv sv;
            sv.t = t;
            sv.d2 = tri_closest_f64(pn, A, Bv, Cv, sv.c, &sv.interior, &sv.near);
            int slot = atomicAdd(&s_ns[wib], 1);
            if (slot < kSurvCap) s_surv[wib][slot] = sv;
          }
        }
      }
  __syncwarp();
  const int ns = s_ns[wib];
  if (lane != 0) return;
  if (ns > kSurvCap) {
    sc->ncon[f] = 0;
    atomicCAS(&sc->status, 0, ST_CAPACITY);
    return;
  }
  int g = -1;
  double gd = 0.0;
  for (int i = 0; i < ns; ++i) {
    const Surv& sv = s_surv[wib][i];
    if (g < 0 || sv.d2 < gd || (sv.d2 == gd && sv.t < s_surv[wib][g].t)) { g = i; gd = sv.d2; }
  }
  int ord[kSurvCap];
  for (int i = 0; i < ns; ++i) {
    int j = i;
    while (j > 0 && s_surv[wib][ord[j - 1]].t > s_surv[wib][i].t) { ord[j] = ord[j - 1]; --j; }
    ord[j] = i;
  }
  int nc = 0;
  int* ctri = sc->tri + (size_t)f * kNoAllocCpn;
  double* cpt = sc->pt + (size_t)f * kNoAllocCpn * 3;
  double* cn = sc->nrm + (size_t)f * kNoAllocCpn * 3;
  double* cg = sc->gap + (size_t)f * kNoAllocCpn;
  for (int oi = 0; oi < ns; ++oi) {
    const Surv& sv = s_surv[wib][ord[oi]];
    double dist = sqrt(sv.d2);
    if (!(dist <= thr)) continue;
    if (!(sv.near || ord[oi] == g)) continue;
    bool dup = false;
    for (int r = 0; r < nc; ++r) {
      double dx = cpt[3 * r] - sv.c[0], dy = cpt[3 * r + 1] - sv.c[1], dz = cpt[3 * r + 2] - sv.c[2];
      if (dx * dx + dy * dy + dz * dz <= 1e-24) { dup = true; break; }   // |c_j - c_i| <= 1e-12 m
    }
    if (dup) continue;
    if (nc >= kNoAllocCpn) { atomicCAS(&sc->status, 0, ST_CAPACITY); break; }
    const double* nf = d.nface + 3 * (size_t)sv.t;
    double nv[3];
    double cmp[3] = {sv.c[0] - pn[0], sv.c[1] - pn[1], sv.c[2] - pn[2]};
    if (sv.interior || dist < 1e-12) { nv[0] = nf[0]; nv[1] = nf[1]; nv[2] = nf[2]; }
    else {
      double sgn = (dot3(nf, cmp) > 0.0) ? 1.0 : -1.0;
      double id = sgn / dist;
      nv[0] = cmp[0] * id; nv[1] = cmp[1] * id; nv[2] = cmp[2] * id;
    }
    ctri[nc] = sv.t;
    cpt[3 * nc] = sv.c[0]; cpt[3 * nc + 1] = sv.c[1]; cpt[3 * nc + 2] = sv.c[2];
    cn[3 * nc] = nv[0]; cn[3 * nc + 1] = nv[1]; cn[3 * nc + 2] = nv[2];
    cg[nc] = dot3(nv, sv.c) - dot3(nv, pn) - p.r_o;
    ++nc;
  }
  sc->ncon[f] = nc;
}

// One CTA: rows of all nodes in (node, triangle) order into the caller's arrays (first cap rows).
__global__ void __launch_bounds__(1024) rows_noalloc_kernel(int n, int cap, NoAllocScratch* sc, int32_t* row_node,
                                                            int32_t* row_tri, double* row_point, double* row_normal,
                                                            double* row_gap, int32_t* n_rows) {
  __shared__ int s_warp[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int per = (n + 1023) / 1024;
  const int f0 = tid * per, f1 = min(f0 + per, n);
  int loc = 0;
  for (int f = f0; f < f1; ++f) loc += sc->ncon[f];
  int v = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) s_warp[w] = v;
  __syncthreads();
  if (w == 0) {
    int x = s_warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    s_warp[lane] = x;
  }
  __syncthreads();
  int row = v - loc + (w > 0 ? s_warp[w - 1] : 0);
  for (int f = f0; f < f1; ++f)
    for (int r = 0; r < sc->ncon[f]; ++r, ++row) {
      if (row >= cap) continue;
      row_node[row] = f;
      row_tri[row] = sc->tri[f * kNoAllocCpn + r];
      for (int c = 0; c < 3; ++c) {
        row_point[3 * row + c] = sc->pt[(f * kNoAllocCpn + r) * 3 + c];
        row_normal[3 * row + c] = sc->nrm[(f * kNoAllocCpn + r) * 3 + c];
      }
      row_gap[row] = sc->gap[f * kNoAllocCpn + r];
    }
  if (tid == 0) {
    sc->n_rows = s_warp[31];
    *n_rows = s_warp[31];
  }
}

}  // namespace accfem

using namespace accfem;

// Internal views of a handle (defined with the handle in api.cu).
bool accfem_internal_views(accfem_handle* h, Params* p, Dev* d, cudaStream_t* stream);
void accfem_internal_set_error(accfem_handle* h, const char* msg);
bool accfem_internal_on_device(accfem_handle* h, const char* who);

namespace {
constexpr int kMaxDevices = 64;
NoAllocScratch* g_scratch_addr[kMaxDevices] = {nullptr};
}  // namespace

extern "C" accfem_status accfem_detect_contacts_noalloc(accfem_handle* h, const double* node_pos, int32_t n_nodes,
                                                        int32_t row_capacity, int32_t* row_node, int32_t* row_tri,
                                                        double* row_point, double* row_normal, double* row_gap,
                                                        int32_t* n_rows, void* stream) {
  if (!h) return ACCFEM_E_INVALID_ARG;
  if (n_nodes < 0 || n_nodes > kNoAllocMaxNodes) {
    accfem_internal_set_error(h, "accfem_detect_contacts_noalloc: n_nodes must be in [0, 4096]");
    return ACCFEM_E_INVALID_ARG;
  }
  if (row_capacity < 0 || (n_nodes > 0 && !node_pos) || !n_rows ||
      (row_capacity > 0 && (!row_node || !row_tri || !row_point || !row_normal || !row_gap))) {
    accfem_internal_set_error(h, "accfem_detect_contacts_noalloc: NULL buffer or negative capacity");
    return ACCFEM_E_INVALID_ARG;
  }
  if (!accfem_internal_on_device(h, "accfem_detect_contacts_noalloc")) return ACCFEM_E_INVALID_ARG;
  Params p;
  Dev d;
  cudaStream_t own;
  if (!accfem_internal_views(h, &p, &d, &own)) return ACCFEM_E_INVALID_ARG;
  cudaStream_t st = stream ? (cudaStream_t)stream : own;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    accfem_internal_set_error(h, "accfem_detect_contacts_noalloc: no current CUDA device");
    return ACCFEM_E_CUDA;
  }
  // once per device, with that device current: the device address of the file-scope scratch
  if (!g_scratch_addr[dev]) {
    void* addr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
    if (e != cudaSuccess || !addr) {
      accfem_internal_set_error(h, cudaGetErrorString(e));
      return ACCFEM_E_CUDA;
    }
    g_scratch_addr[dev] = (NoAllocScratch*)addr;
  }
  NoAllocScratch* sc = g_scratch_addr[dev];
  {
    cudaError_t e = cudaMemsetAsync(&sc->status, 0, sizeof(int), st);
    if (e != cudaSuccess) {
      accfem_internal_set_error(h, cudaGetErrorString(e));
      return ACCFEM_E_CUDA;
    }
  }
  if (n_nodes > 0) detect_noalloc_kernel<<<(n_nodes + 3) / 4, 128, 0, st>>>(p, d, node_pos, n_nodes, sc);
  rows_noalloc_kernel<<<1, 1024, 0, st>>>(n_nodes, row_capacity, sc, row_node, row_tri, row_point, row_normal, row_gap,
                                          n_rows);
  int res[2] = {0, 0};
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(res, &sc->status, 2 * sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    accfem_internal_set_error(h, "accfem_detect_contacts_noalloc: CUDA error");
    return ACCFEM_E_CUDA;
  }
  if (res[0] != 0 || res[1] > row_capacity) {
    accfem_internal_set_error(h, res[0] != 0 ? "accfem_detect_contacts_noalloc: a node has more than 64 triangles for "
                                               "the exact test or more than 16 rows"
                                             : "accfem_detect_contacts_noalloc: more rows than row_capacity");
    return ACCFEM_E_CONTACT_CAPACITY;
  }
  return ACCFEM_OK;
}
