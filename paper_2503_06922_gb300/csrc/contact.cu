// Contact-space solve of the QP of Eq. 23 (equivalently the MLCP of Eq. 22) for one Newton step.
//
// With X = K^{-1} A^T (RHS columns 1..m) and dx_free = -K^{-1} g (column 0), the step is
// dx = dx_free - X y where y >= 0 solves the LCP
//     w = W y + q >= 0,  y >= 0,  y^T w = 0,     W = A X,  q = b - A dx_free,
// w being the slack b - A dx of Eq. 8 and y the contact forces of Eq. 11-12.  W is symmetric
// positive semi-definite; with the contact compliance 1e-12 max(diag W) added to its diagonal it is
// positive definite, so the solution is unique.
// It is found exactly by the primal active-set method below; every subproblem W_PP z_P = -q_P is
// solved in FP64 by Gauss-Jordan over the whole CTA.  One CTA of 1024 threads; W and the
// elimination matrix live in global memory (L2 resident).
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

__device__ __forceinline__ int block_min_int_unused(int v, int* s_ired) {
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

// (value, index) minimum over the block; ties resolved to the lowest index.
__device__ __forceinline__ void block_argmin(double& v, int& idx, double* s_red, int* s_ired) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_xor_sync(0xffffffffu, v, o);
    int oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov < v || (ov == v && oi < idx)) { v = ov; idx = oi; }
  }
  __syncthreads();
  if (lane == 0) { s_red[w] = v; s_ired[w] = idx; }
  __syncthreads();
  if (w == 0) {
    double x = lane < (blockDim.x >> 5) ? s_red[lane] : 1.0e300;
    int xi = lane < (blockDim.x >> 5) ? s_ired[lane] : 0x7fffffff;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_xor_sync(0xffffffffu, x, o);
      int oi = __shfl_xor_sync(0xffffffffu, xi, o);
      if (ov < x || (ov == x && oi < xi)) { x = ov; xi = oi; }
    }
    if (lane == 0) { s_red[32] = x; s_ired[32] = xi; }
  }
  __syncthreads();
  v = s_red[32];
  idx = s_ired[32];
}

// Solves W_PP z_P = -q_P for the rows flagged in inP (Gauss-Jordan over the CTA, FP64) and writes
// z into d.w (0 outside P).  Returns the size of P, or -1 on a non-positive pivot.
__device__ int solve_on_set(const Dev& d, int m, int* s_np) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __syncthreads();
  if (tid == 0) {
    int np = 0;
    for (int i = 0; i < m; ++i)
      if (d.inP[i]) d.plist[np++] = i;
    *s_np = np;
  }
  __syncthreads();
  const int np = *s_np;
  const int ldg = np + 1;
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
    const int wdt = ldg - k - 1;
    for (int idx = tid; idx < np * wdt; idx += nt) {
      int r = idx / wdt, c = k + 1 + idx % wdt;
      if (r == k) continue;
      d.gj[(size_t)r * ldg + c] = fma(-d.gj[(size_t)r * ldg + k], d.gj[(size_t)k * ldg + c], d.gj[(size_t)r * ldg + c]);
    }
  }
  __syncthreads();
  if (!spd) return -1;
  for (int i = tid; i < m; i += nt) d.w[i] = 0.0;
  __syncthreads();
  for (int r = tid; r < np; r += nt) d.w[d.plist[r]] = d.gj[(size_t)r * ldg + np];
  __syncthreads();
  return np;
}

// LCP by a primal active-set method for the bound-constrained QP min 1/2 y^T W y + q^T y, y >= 0
// (the Lawson-Hanson NNLS scheme with W SPD): keep y feasible with y_P > 0; add the row of most
// negative w = W y + q; when the subproblem solution z_P has non-positive entries, step from y
// towards z up to the first bound and release the rows that reach zero.  Finite for SPD W; starts
// from the rows active in the previous Newton iteration.  d.w holds z, d.y holds y.
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
    d.inP[i] = d.init_act[i] > 0 ? 1 : 0;
    d.y[i] = 0.0;
  }
  __syncthreads();
  // contact compliance eps = 1e-12 max_i W_ii on the diagonal: rows of one node are linearly
  // dependent where four or more wall faces meet, which leaves W singular without it
  double wd = 0.0;
  for (int i = tid; i < m; i += nt) wd = fmax(wd, d.W[(size_t)i * m + i]);
  wd = block_max(wd, s_red);
  for (int i = tid; i < m; i += nt) d.W[(size_t)i * m + i] += 1e-12 * wd;
  double qmax = 0.0;
  for (int i = tid; i < m; i += nt) qmax = fmax(qmax, fabs(d.q[i]));
  qmax = block_max(qmax, s_red);
  const double tol_w = p.lcp_tol * fmax(qmax, 1e-300);
  int solves = 0;
  bool done = false, fail = false;
  // ---- feasible start: drop warm rows until the subproblem solution is positive
  for (;;) {
    if (solves >= p.max_lcp_iters) break;
    int np = solve_on_set(d, m, &s_np);
    ++solves;
    if (np < 0) { fail = true; break; }
    int nneg = 0;
    for (int i = tid; i < m; i += nt)
      if (d.inP[i] && !(d.w[i] > 0.0)) { d.inP[i] = 0; ++nneg; }
    nneg = block_sum_int(nneg, s_ired);
    if (nneg == 0) {
      for (int i = tid; i < m; i += nt) d.y[i] = d.w[i];
      break;
    }
  }
  // ---- main loop
  while (!fail && solves < p.max_lcp_iters) {
    __syncthreads();
    // w = W y + q outside P; most negative entry
    double best = 1.0e300;
    int bi = 0x7fffffff;
    for (int i = tid; i < m; i += nt) {
      if (d.inP[i]) continue;
      double s = d.q[i];
      for (int j = 0; j < m; ++j)
        if (d.inP[j]) s = fma(d.W[(size_t)i * m + j], d.y[j], s);
      if (s < -tol_w && (s < best || (s == best && i < bi))) { best = s; bi = i; }
    }
    block_argmin(best, bi, s_red, s_ired);
    if (bi == 0x7fffffff) { done = true; break; }
    if (tid == 0) d.inP[bi] = 1;
    // inner loop: restore y_P > 0
    for (;;) {
      if (solves >= p.max_lcp_iters) break;
      int np = solve_on_set(d, m, &s_np);
      ++solves;
      if (np < 0) { fail = true; break; }
      // alpha = min over P with z_i <= 0 of y_i / (y_i - z_i)
      double amin = 1.0e300;
      int dummy = 0;
      for (int i = tid; i < m; i += nt)
        if (d.inP[i] && !(d.w[i] > 0.0)) {
          double yi = d.y[i], zi = d.w[i];
          double a = (yi - zi) > 0.0 ? yi / (yi - zi) : 0.0;
          amin = fmin(amin, a);
        }
      block_argmin(amin, dummy, s_red, s_ired);
      if (amin >= 1.0e300) {
        for (int i = tid; i < m; i += nt) d.y[i] = d.w[i];
        break;
      }
      double ymax = 0.0;
      for (int i = tid; i < m; i += nt) {
        if (d.inP[i]) {
          double v = d.y[i] + amin * (d.w[i] - d.y[i]);
          d.y[i] = v;
          ymax = fmax(ymax, v);
        }
      }
      ymax = block_max(ymax, s_red);
      const double tol_y = p.lcp_tol * fmax(ymax, 1e-300);
      for (int i = tid; i < m; i += nt)
        if (d.inP[i] && d.y[i] <= tol_y) { d.inP[i] = 0; d.y[i] = 0.0; }
    }
  }
  __syncthreads();
  if (tid == 0) {
    ctl->lcp_pivots += solves;
    if (fail) atomicCAS(&ctl->status, 0, ST_NOT_SPD);
    else if (!done) atomicCAS(&ctl->status, 0, ST_TIMEOUT);
    int na = 0;
    for (int i = 0; i < m; ++i) {
      const bool a = d.inP[i] && d.y[i] > 0.0;
      d.p_act[i] = a ? 1 : 0;
      if (a) d.plist[na++] = i;
      else d.y[i] = 0.0;
    }
    ctl->n_active = na;
  }
}

}  // namespace accfem
