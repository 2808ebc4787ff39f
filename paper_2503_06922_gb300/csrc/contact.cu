// Contact-space solve of the QP of Eq. 23 (equivalently the MLCP of Eq. 22) for one Newton step.
//
// With X = K^{-1} A^T (RHS columns 1..m) and dx_free = -K^{-1} g (column 0), the step is
// dx = dx_free - X y where y >= 0 solves the LCP
//     w = W y + q >= 0,  y >= 0,  y^T w = 0,     W = A X,  q = b - A dx_free,
// w being the slack b - A dx of Eq. 8 and y the contact forces of Eq. 11-12.  W is symmetric
// positive semi-definite; with the contact compliance 1e-12 max(diag W) added to its diagonal it is
// positive definite, so the solution is unique.
// It is found exactly by principal pivoting: from the guess P = {q_i < 0}, solve W_PP y_P = -q_P
// in FP64 (Gauss-Jordan over the whole CTA), test the complementary variables, flip every
// infeasible index (block pivoting, Judice-Pires); when the count of infeasible indices stops
// falling for 3 rounds, flip only the least such index (Murty's rule, finite for P-matrices).
// One CTA of 1024 threads; W and the elimination matrix live in global memory (L2 resident).
#include "common.cuh"

namespace accfem {

__device__ __forceinline__ double block_max(double v, double* s_red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) s_red[w] = v;
  __syncthreads();
  if (w == 0) {
    double x = lane < (blockDim.x >> 5) ? s_red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) s_red[32] = x;
  }
  __syncthreads();
  return s_red[32];
}

__device__ __forceinline__ int block_sum_int(int v, int* s_ired) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) s_ired[w] = v;
  __syncthreads();
  if (w == 0) {
    int x = lane < (blockDim.x >> 5) ? s_ired[lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) s_ired[32] = x;
  }
  __syncthreads();
  return s_ired[32];
}

__device__ __forceinline__ int block_min_int(int v, int* s_ired) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) s_ired[w] = v;
  __syncthreads();
  if (w == 0) {
    int x = lane < (blockDim.x >> 5) ? s_ired[lane] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = min(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) s_ired[32] = x;
  }
  __syncthreads();
  return s_ired[32];
}

__global__ void __launch_bounds__(1024) contact_kernel(Params p, Dev d) {
  __shared__ double s_red[33];
  __shared__ int s_ired[33];
  __shared__ int s_np;
  Ctl* ctl = d.ctl;
  if (ctl->status != 0 || ctl->converged) return;
  const int m = ctl->m;
  const int tid = threadIdx.x, nt = blockDim.x;
  const size_t ld = p.nrhs_cap;
  if (m == 0) {
    if (tid == 0) { ctl->n_active = 0; }
    return;
  }
  // ---- W and q
  for (int idx = tid; idx < m * m; idx += nt) {
    int i = idx / m, j = idx % m;
    int fi = d.c_node[i];
    const double* n = d.c_n + 3 * i;
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) s = fma(n[c], d.B[((size_t)fi * 6 + c) * ld + 1 + j], s);
    d.W[(size_t)i * m + j] = s;
  }
  for (int i = tid; i < m; i += nt) {
    int fi = d.c_node[i];
    const double* n = d.c_n + 3 * i;
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) s = fma(n[c], d.B[((size_t)fi * 6 + c) * ld], s);
    d.q[i] = d.c_gap[i] - s;
    d.inP[i] = d.q[i] < 0.0 ? 1 : 0;
  }
  __syncthreads();
  // contact compliance eps = 1e-12 max_i W_ii on the diagonal: rows of one node are linearly
  // dependent where four or more wall faces meet, which leaves W singular without it
  double wd = 0.0;
  for (int i = tid; i < m; i += nt) wd = fmax(wd, d.W[(size_t)i * m + i]);
  wd = block_max(wd, s_red);
  for (int i = tid; i < m; i += nt) d.W[(size_t)i * m + i] += 1e-12 * wd;
  __syncthreads();
  double qmax = 0.0;
  for (int i = tid; i < m; i += nt) qmax = fmax(qmax, fabs(d.q[i]));
  qmax = block_max(qmax, s_red);
  const double tol_w = p.lcp_tol * fmax(qmax, 1e-300);
  int best = 0x7fffffff, stall = 0, pivots = 0;
  bool done = false;
  for (int it = 0; it < p.max_lcp_iters; ++it) {
    // ---- P list
    if (tid == 0) {
      int np = 0;
      for (int i = 0; i < m; ++i)
        if (d.inP[i]) d.plist[np++] = i;
      s_np = np;
    }
    __syncthreads();
    const int np = s_np;
    const int ldg = np + 1;
    // ---- [W_PP | -q_P] and Gauss-Jordan
    for (int idx = tid; idx < np * ldg; idx += nt) {
      int r = idx / ldg, c = idx % ldg;
      int i = d.plist[r];
      d.gj[idx] = (c < np) ? d.W[(size_t)i * m + d.plist[c]] : -d.q[i];
    }
    bool spd = true;
    for (int k = 0; k < np; ++k) {
      __syncthreads();
      double akk = d.gj[(size_t)k * ldg + k];
      if (!(akk > 0.0)) { spd = false; break; }
      double rp = 1.0 / akk;
      for (int c = k + 1 + tid; c < ldg; c += nt) d.gj[(size_t)k * ldg + c] *= rp;
      __syncthreads();
      const int w = ldg - k - 1;
      for (int idx = tid; idx < np * w; idx += nt) {
        int r = idx / w, c = k + 1 + idx % w;
        if (r == k) continue;
        d.gj[(size_t)r * ldg + c] = fma(-d.gj[(size_t)r * ldg + k], d.gj[(size_t)k * ldg + c], d.gj[(size_t)r * ldg + c]);
      }
    }
    __syncthreads();
    if (!spd) {
      if (tid == 0) atomicCAS(&ctl->status, 0, ST_NOT_SPD);
      return;
    }
    for (int i = tid; i < m; i += nt) d.y[i] = 0.0;
    __syncthreads();
    for (int r = tid; r < np; r += nt) d.y[d.plist[r]] = d.gj[(size_t)r * ldg + np];
    __syncthreads();
    double ymax = 0.0;
    for (int i = tid; i < m; i += nt) ymax = fmax(ymax, fabs(d.y[i]));
    ymax = block_max(ymax, s_red);
    const double tol_y = p.lcp_tol * fmax(ymax, 1e-300);
    // ---- complementary variables, infeasible set
    int nbad = 0, first = 0x7fffffff;
    for (int i = tid; i < m; i += nt) {
      bool bad;
      if (d.inP[i]) {
        bad = d.y[i] < -tol_y;
        d.w[i] = 0.0;
      } else {
        double s = d.q[i];
        for (int r = 0; r < np; ++r) s = fma(d.W[(size_t)i * m + d.plist[r]], d.y[d.plist[r]], s);
        d.w[i] = s;
        bad = s < -tol_w;
      }
      if (bad) { ++nbad; first = min(first, i); }
      d.gj[(size_t)np * ldg + i] = bad ? 1.0 : 0.0;   // scratch flag row (past the system)
    }
    nbad = block_sum_int(nbad, s_ired);
    first = block_min_int(first, s_ired);
    if (nbad == 0) { done = true; break; }
    ++pivots;
    if (nbad < best) { best = nbad; stall = 0; } else { ++stall; }
    const bool murty = stall >= 3;
    for (int i = tid; i < m; i += nt) {
      bool bad = d.gj[(size_t)np * ldg + i] != 0.0;
      if (murty ? (i == first) : bad) d.inP[i] = 1 - d.inP[i];
    }
    __syncthreads();
  }
  if (tid == 0) {
    ctl->lcp_pivots += pivots;
    if (!done) atomicCAS(&ctl->status, 0, ST_TIMEOUT);
    int na = 0;
    for (int i = 0; i < m; ++i)
      if (d.inP[i] && d.y[i] != 0.0) d.plist[na++] = i;
    ctl->n_active = na;
  }
}

}  // namespace accfem
