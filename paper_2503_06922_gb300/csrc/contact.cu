// Contact-space solve of the QP of Eq. 23 (equivalently the MLCP of Eq. 22) for one Newton step.
//
// With X = K^{-1} A^T (RHS columns 1..m) and dx_free = -K^{-1} g (column 0), the step is
// dx = dx_free - X y where y >= 0 solves the LCP
//     w = W y + q >= 0,  y >= 0,  y^T w = 0,     W = A X,  q = b - A dx_free,
// w being the slack b - A dx of Eq. 8 and y the contact forces of Eq. 11-12.  W is symmetric
// positive semi-definite; with the contact compliance 1e-12 max(diag W) added to its diagonal it is
// positive definite, so the solution is unique.
// It is found exactly by the primal active-set method below; every subproblem W_PP z_P = -q_P is
// solved in FP64 by Gauss-Jordan over the whole CTA.  One CTA per instance; the columns of W that
// the active set touches are formed on demand in global memory (L2 resident), the Gauss-Jordan
// matrix of subproblems up to kLcpSmemGJ rows lives in shared memory.
#include "batch.cuh"

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

constexpr int kLcpThreads = 256;
constexpr int kLcpSmemRows = kMaxWorking;   // working-set rows kept in shared memory
constexpr int kLcpSmemGJ = 48;         // active rows solved in shared memory (else in global memory)

struct LcpShared {
  double q[kLcpSmemRows], y[kLcpSmemRows], z[kLcpSmemRows];
  int inP[kLcpSmemRows], wcol[kLcpSmemRows], plist[kLcpSmemRows];
  double gj[kLcpSmemGJ * (kLcpSmemGJ + 1)];
  double prow[kLcpSmemRows + 1];         // scaled pivot row of the Gauss-Jordan step
  double red[33];
  int ired[33];
  int np;
};

// Forms column j of W = A X (with the compliance eps on its diagonal) for every active slot j whose
// column is not formed yet: W_ij = n_i . X_j[node_i] over the working-set slots i (row wrow[i]).
// W is symmetric, so the rows of the active columns give every entry the active-set method reads.
// W: m x m row-major, in shared or global memory.
__device__ void ensure_columns(const Dev& d, LcpShared& S, int m, size_t ld, double eps_w, double* W) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __syncthreads();
  // a thread owns rows i (its node's RHS entries and normal loaded once) and forms their entries of
  // every new column; the RHS columns are read-only here, so the loads of different columns overlap
  for (int i = tid; i < m; i += nt) {
    const int row = d.wrow[i];
    const int fi = d.c_node[row], fi2 = d.c_node2[row];
    const double n0 = d.c_w1[3 * row], n1 = d.c_w1[3 * row + 1], n2 = d.c_w1[3 * row + 2];
    const double* b0 = d.B + ((size_t)fi * 6) * ld + 1;
    const double* b1 = b0 + ld;
    const double* b2 = b1 + ld;
    if (fi2 < 0) {
      for (int a = 0; a < S.np; ++a) {
        const int j = S.plist[a];
        if (S.wcol[j]) continue;
        double s = 0.0;
        s = fma(n0, __ldg(b0 + j), s);
        s = fma(n1, __ldg(b1 + j), s);
        s = fma(n2, __ldg(b2 + j), s);
        if (i == j) s += eps_w;
        W[(size_t)i * m + j] = s;
      }
    } else {                                       // a segment row also weighs the element's near node
      const double m0 = d.c_w2[3 * row], m1 = d.c_w2[3 * row + 1], m2 = d.c_w2[3 * row + 2];
      const double* c0 = d.B + ((size_t)fi2 * 6) * ld + 1;
      const double* c1 = c0 + ld;
      const double* c2 = c1 + ld;
      for (int a = 0; a < S.np; ++a) {
        const int j = S.plist[a];
        if (S.wcol[j]) continue;
        double s = 0.0;
        s = fma(n0, __ldg(b0 + j), s);
        s = fma(n1, __ldg(b1 + j), s);
        s = fma(n2, __ldg(b2 + j), s);
        s = fma(m0, __ldg(c0 + j), s);
        s = fma(m1, __ldg(c1 + j), s);
        s = fma(m2, __ldg(c2 + j), s);
        if (i == j) s += eps_w;
        W[(size_t)i * m + j] = s;
      }
    }
  }
  __syncthreads();
  for (int a = tid; a < S.np; a += nt) S.wcol[S.plist[a]] = 1;
  __syncthreads();
}

// Rebuilds the active list from the flags (warp 0, ballot compaction; rows in increasing order).
__device__ void rebuild_plist(LcpShared& S, int m) {
  __syncthreads();
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int np = 0;
    for (int i0 = 0; i0 < m; i0 += 32) {
      const int i = i0 + lane;
      const bool in = i < m && S.inP[i];
      const unsigned mk = __ballot_sync(0xffffffffu, in);
      if (in) S.plist[np + __popc(mk & ((1u << lane) - 1u))] = i;
      np += __popc(mk);
    }
    if (lane == 0) S.np = np;
  }
  __syncthreads();
}

// Solves W_PP z_P = -q_P for the active list (Gauss-Jordan with 2x2 block pivots over the CTA, FP64;
// shared memory for up to kLcpSmemGJ rows) and writes z (0 outside P).  Returns false on a
// non-positive pivot.
__device__ bool solve_on_set(const Dev& d, LcpShared& S, int m, const double* W) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int np = S.np;
  const int ldg = np + 1;
  double* G = np <= kLcpSmemGJ ? S.gj : d.gj;
  for (int idx = tid; idx < np * ldg; idx += nt) {
    int r = idx / ldg, c = idx % ldg;
    int i = S.plist[r];
    G[idx] = (c < np) ? W[(size_t)i * m + S.plist[c]] : -S.q[i];
  }
  // 2x2 block pivots (rows k, k + 1): the block's inverse from its determinant (one reciprocal for
  // two rows), both pivot rows scaled by it, every other row updated by both at once; a last single
  // row takes a scalar pivot.  The block is SPD exactly when its two scalar pivots (a, det / a) are
  // positive.
  double* q1 = S.z;                                // second scaled pivot row (S.z is written at the end)
  const int step = ldg <= kLcpSmemRows ? 2 : 1;    // (S.z holds kLcpSmemRows entries)
  for (int k = 0; k < np; k += step) {
    __syncthreads();
    if (k + 1 == np || step == 1) {
      const double akk = G[(size_t)k * ldg + k];
      if (!(akk > 0.0)) return false;
      if (tid < 32) {
        const double rp = __drcp_rn(akk);
        for (int c = k + 1 + tid; c < ldg; c += 32) S.prow[c] = G[(size_t)k * ldg + c] * rp;
      }
      __syncthreads();
      const int wdt = ldg - k - 1;
      for (int idx = tid; idx < np * wdt; idx += nt) {
        int r = idx / wdt, c = k + 1 + idx % wdt;
        G[(size_t)r * ldg + c] = r == k ? S.prow[c] : fma(-G[(size_t)r * ldg + k], S.prow[c], G[(size_t)r * ldg + c]);
      }
      continue;
    }
    const double a = G[(size_t)k * ldg + k], b = G[(size_t)k * ldg + k + 1];
    const double b2 = G[(size_t)(k + 1) * ldg + k], cc = G[(size_t)(k + 1) * ldg + k + 1];
    const double det = fma(a, cc, -(b * b2));
    if (!(a > 0.0) || !(det > 0.0)) return false;
    // the two scaled pivot rows, Binv [a_k; a_k+1] (one reciprocal per block): the first by warp 0,
    // the second by warp 1, each from the two entries of Binv it uses (a warp's FP64 instruction
    // holds its SMSP's FP64 pipe for 64 cycles, so the two rows run on two SMSPs at once)
    if (tid < 64) {
      const bool second = tid >= 32;
      const double rd = __drcp_rn(det);
      const double e0 = (second ? -b2 : cc) * rd, e1 = (second ? a : -b) * rd;
      double* dst = second ? q1 : S.prow;
      for (int c = k + 2 + (tid & 31); c < ldg; c += 32) {
        const double g0 = G[(size_t)k * ldg + c], g1 = G[(size_t)(k + 1) * ldg + c];
        dst[c] = fma(e0, g0, e1 * g1);
      }
    }
    __syncthreads();
    const int wdt = ldg - k - 2;
    for (int idx = tid; idx < np * wdt; idx += nt) {
      int r = idx / wdt, c = k + 2 + idx % wdt;
      double v;
      if (r == k) v = S.prow[c];
      else if (r == k + 1) v = q1[c];
      else v = fma(-G[(size_t)r * ldg + k], S.prow[c], fma(-G[(size_t)r * ldg + k + 1], q1[c], G[(size_t)r * ldg + c]));
      G[(size_t)r * ldg + c] = v;
    }
  }
  __syncthreads();
  for (int i = tid; i < m; i += nt) S.z[i] = 0.0;
  __syncthreads();
  for (int r = tid; r < np; r += nt) S.z[S.plist[r]] = G[(size_t)r * ldg + np];
  __syncthreads();
  return true;
}

// OSQP's ADMM (Stellato et al., 2020: the solver the paper uses for Eq. 23) on the contact-space QP
// min 1/2 y^T W y + q^T y, y >= 0 over the working set (OSQP's P = W, constraint matrix I, l = 0,
// u = inf), with step sizes sigma = 1e-6, rho = 0.1 max(diag W) and relaxation alpha = 1.6:
//   (W + (sigma + rho) I) yt = sigma y - q + rho z - lam
//   y <- alpha yt + (1 - alpha) y,  zh = alpha yt + (1 - alpha) z,
//   z <- max(zh + lam / rho, 0),    lam <- lam + rho (zh - z),
// stopped when |y - z| <= 1e-3 max(|y|, |z|) and |W y + q + lam| <= 1e-3 max(|W y|, |lam|, |q|)
// (infinity norms, tested every 10 iterations) or after p.admm_iters iterations.  Its only product
// is the guess of the free rows (z > -lam) that starts the exact FP64 active-set method, which
// polishes it to the unique solution; so the ADMM runs in FP32, where a warp instruction costs one
// issue cycle instead of the FP64 pipe's 64: W + (sigma + rho) I (condition number below about 10 m,
// since rho is a tenth of the largest diagonal entry) is inverted once by Gauss-Jordan in shared
// memory (global memory past kAdmmSmemRows rows), an iteration is one product with the inverse (tpr
// threads per row, the rows' updates in parallel) and the projection.  A non-positive FP32 pivot drops the guess: the exact method then
// starts from the empty set.
// Partial dot product of column i of the symmetric m x m matrix A (row-major) with x over the
// entries j = t, t + tpr, ...; four independent FP32 sums, so that the loads run ahead of the FMAs.
__device__ __forceinline__ float col_dot(const float* A, const float* x, int m, int i, int t, int tpr) {
  float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
  const float* a = A + i;
  int j = t;
  for (; j + 3 * tpr < m; j += 4 * tpr) {
    s0 = fmaf(a[j * m], x[j], s0);
    s1 = fmaf(a[(j + tpr) * m], x[j + tpr], s1);
    s2 = fmaf(a[(j + 2 * tpr) * m], x[j + 2 * tpr], s2);
    s3 = fmaf(a[(j + 3 * tpr) * m], x[j + 3 * tpr], s3);
  }
  for (; j < m; j += tpr) s0 = fmaf(a[j * m], x[j], s0);
  return (s0 + s1) + (s2 + s3);
}

__device__ void admm_guess(const Params& p, const Dev& d, LcpShared& S, int m, size_t ld, double eps_w, int* iters) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
  for (int i = tid; i < m; i += nt) S.inP[i] = 1;
  rebuild_plist(S, m);
  ensure_columns(d, S, m, ld, eps_w, d.W);      // every column of W over the working set (FP64)
  double wd = 0.0;
  for (int i = tid; i < m; i += nt) wd = fmax(wd, d.W[(size_t)i * m + i]);
  wd = block_max(wd, S.red);
  const float sigma = 1.0e-6f, alpha = 1.6f, eps_rel = 1.0e-3f;
  const float rho = (float)(0.1 * wd), irho = 1.0f / rho;
  // FP32 state in the shared Gauss-Jordan area (unused until the polish)
  float* fq = reinterpret_cast<float*>(S.gj);
  float* fy = fq + kLcpSmemRows;
  float* fz = fy + kLcpSmemRows;
  float* fl = fz + kLcpSmemRows;
  float* frv = fl + kLcpSmemRows;
  float* frow = frv + kLcpSmemRows;             // scaled pivot row
  float* fcol = frow + kLcpSmemRows;            // pivot column
  // (W + (sigma + rho) I)^-1, m x m row-major: in the launch's dynamic shared memory when it fits
  // (kernels launched for the ADMM solver), else in global memory; W in FP32 for the residual test
  extern __shared__ float s_admm[];
  unsigned dyn_bytes;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_bytes));
  const bool in_smem = (size_t)m * m * sizeof(float) <= dyn_bytes;
  float* G = in_smem ? s_admm : reinterpret_cast<float*>(d.gj);
  float* W32 = reinterpret_cast<float*>(d.gj) + (in_smem ? 0 : (size_t)m * m);
  for (int i = wid; i < m; i += nw)
    for (int j = lane; j < m; j += 32) {
      const double w = d.W[(size_t)i * m + j];
      W32[(size_t)i * m + j] = (float)w;
      G[(size_t)i * m + j] = (float)(i == j ? w + (1.0e-6 + 0.1 * wd) : w);
    }
  for (int i = tid; i < m; i += nt) { fq[i] = (float)S.q[i]; fy[i] = 0.0f; fz[i] = 0.0f; fl[i] = 0.0f; }
  bool ok = true;
  for (int k = 0; k < m; ++k) {
    __syncthreads();
    const float akk = G[(size_t)k * m + k];
    if (!(akk > 0.0f)) { ok = false; break; }   // the same value for every thread
    if (tid < 32) {
      const float pk = 1.0f / akk;
      for (int j = tid; j < m; j += 32) frow[j] = j == k ? pk : G[(size_t)k * m + j] * pk;
    }
    for (int i = tid; i < m; i += nt) fcol[i] = G[(size_t)i * m + k];
    __syncthreads();
    const float pk = frow[k];
    for (int i = wid; i < m; i += nw) {
      float* gi = G + (size_t)i * m;
      const float ci = fcol[i];
      for (int j = lane; j < m; j += 32) {
        if (i == k) gi[j] = frow[j];
        else if (j == k) gi[j] = -ci * pk;
        else gi[j] = fmaf(-ci, frow[j], gi[j]);
      }
    }
  }
  __syncthreads();
  int it = 0;
  if (ok) {
    // tpr threads per row (a power of two dividing 32, with nt / tpr >= m when m is small)
    int tpr = 1;
    while (tpr < 32 && (nt / (2 * tpr)) >= m) tpr *= 2;
    const int g = tid / tpr, t = tid % tpr, ng = nt / tpr;
    while (it < p.admm_iters) {
      ++it;
      for (int i = tid; i < m; i += nt) frv[i] = ((sigma * fy[i] - fq[i]) + rho * fz[i]) - fl[i];
      __syncthreads();
      for (int i0 = 0; i0 < m; i0 += ng) {       // the same trip count for every thread
        const int i = i0 + g;
        float s = i < m ? col_dot(G, frv, m, i, t, tpr) : 0.0f;   // (G rv)_i, G symmetric
        for (int o = tpr >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (i < m && t == 0) {
          const float zh = alpha * s + (1.0f - alpha) * fz[i];
          const float zn = fmaxf(zh + fl[i] * irho, 0.0f);
          fy[i] = alpha * s + (1.0f - alpha) * fy[i];
          fl[i] = fl[i] + rho * (zh - zn);
          fz[i] = zn;
        }
      }
      __syncthreads();
      if (it % 10 == 0) {
        float rpri = 0.0f, rdua = 0.0f, ym = 0.0f, wym = 0.0f, lm = 0.0f, qm = 0.0f;
        for (int i0 = 0; i0 < m; i0 += ng) {
          const int i = i0 + g;
          float s = i < m ? col_dot(W32, fy, m, i, t, tpr) : 0.0f;   // (W y)_i
          for (int o = tpr >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          if (i < m && t == 0) {
            rpri = fmaxf(rpri, fabsf(fy[i] - fz[i]));
            rdua = fmaxf(rdua, fabsf(s + fq[i] + fl[i]));
            ym = fmaxf(ym, fmaxf(fabsf(fy[i]), fabsf(fz[i])));
            wym = fmaxf(wym, fabsf(s));
            lm = fmaxf(lm, fabsf(fl[i]));
            qm = fmaxf(qm, fabsf(fq[i]));
          }
        }
        // the six maxima over the block in one pass
        float v[6] = {rpri, rdua, ym, wym, lm, qm};
#pragma unroll
        for (int k = 0; k < 6; ++k)
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v[k] = fmaxf(v[k], __shfl_xor_sync(0xffffffffu, v[k], o));
        float* sred = reinterpret_cast<float*>(S.red);   // 66 floats
        if (lane == 0)
#pragma unroll
          for (int k = 0; k < 6; ++k) sred[k * 8 + wid] = v[k];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          float x = 0.0f;
          for (int w2 = 0; w2 < nw; ++w2) x = fmaxf(x, sred[k * 8 + w2]);
          v[k] = x;
        }
        __syncthreads();
        if (v[0] <= eps_rel * v[2] && v[1] <= eps_rel * fmaxf(fmaxf(v[3], v[4]), v[5])) break;
      }
    }
  }
  for (int i = tid; i < m; i += nt) {
    S.inP[i] = (ok && fz[i] > -fl[i]) ? 1 : 0;
    S.y[i] = 0.0;
  }
  __syncthreads();
  *iters = it;
}

// LCP by a primal active-set method for the bound-constrained QP min 1/2 y^T W y + q^T y, y >= 0
// (the Lawson-Hanson NNLS scheme with W SPD): keep y feasible with y_P > 0; add the row of most
// negative w = W y + q; when the subproblem solution z_P has non-positive entries, step from y
// towards z up to the first bound and release the rows that reach zero.  Finite for SPD W; starts
// from the rows active in the previous Newton iteration.  The LCP runs over the working set (slot i
// = row wrow[i], column 1 + i of the RHS); rows outside it get y = 0 and are checked against the
// step afterwards (step kernel).
__device__ __forceinline__ void contact_body(const Params& p, const Dev& d) {
  __shared__ LcpShared S;
  Ctl* ctl = d.ctl;
  if (ctl->status != 0 || ctl->converged) return;
  const int m = ctl->mc;
  const int tid = threadIdx.x, nt = blockDim.x;
  const size_t ld = p.nrhs_cap;
  for (int r = tid; r < ctl->m; r += nt)
    if (d.rslot[r] < 0) d.y[r] = 0.0;
  if (m == 0) {
    if (tid == 0) {
      ctl->n_active = 0;
      ctl->same_active = ctl->n_active_prev == 0 ? 1 : 0;
    }
    return;
  }
  if (m > kLcpSmemRows) {
    if (tid == 0) flag_capacity(ctl, CAP_LCP_ROWS);
    return;
  }
  // ---- q = b - A dx_free; compliance from the largest W_ii
  double wd = 0.0, qmax = 0.0;
  for (int i = tid; i < m; i += nt) {
    const int row = d.wrow[i];
    const int fi = d.c_node[row], fi2 = d.c_node2[row];
    const double* n = d.c_w1 + 3 * row;
    double s = 0.0, wii = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      s = fma(n[c], d.B[((size_t)fi * 6 + c) * ld], s);
      wii = fma(n[c], d.B[((size_t)fi * 6 + c) * ld + 1 + i], wii);
    }
    if (fi2 >= 0) {
      const double* n2 = d.c_w2 + 3 * row;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        s = fma(n2[c], d.B[((size_t)fi2 * 6 + c) * ld], s);
        wii = fma(n2[c], d.B[((size_t)fi2 * 6 + c) * ld + 1 + i], wii);
      }
    }
    const int fl = d.init_flag[row];
    S.q[i] = d.c_gap[row] - s;
    S.y[i] = 0.0;
    S.wcol[i] = 0;
    // the start: the rows active in the previous iteration, or the primal ADMM's guess
    S.inP[i] = p.lcp_mode == kLcpPrimalAdmm ? (d.pa_guess[row] ? 1 : 0) : ((fl > 0 && (fl & RF_ACTIVE)) ? 1 : 0);
    wd = fmax(wd, wii);
    qmax = fmax(qmax, fabs(S.q[i]));
  }
  wd = block_max(wd, S.red);
  qmax = block_max(qmax, S.red);
  const double eps_w = 1e-12 * wd;
  const double tol_w = p.lcp_tol * fmax(qmax, 1e-300);
  int solves = 0;
  bool done = false, fail = false;
  int admm_it = 0;
  if (p.lcp_mode == kLcpAdmm) admm_guess(p, d, S, m, ld, eps_w, &admm_it);
  // W in the launch's dynamic shared memory when it fits (kernels launched with it), except after
  // the contact-space ADMM, whose inverse holds that memory and which formed W in global memory
  extern __shared__ __align__(16) double s_wdyn[];
  unsigned dyn_bytes;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn_bytes));
  double* W = (p.lcp_mode != kLcpAdmm && (size_t)m * m * sizeof(double) <= dyn_bytes) ? s_wdyn : d.W;
  // ---- feasible start: drop warm rows until the subproblem solution is positive
  while (!fail) {
    if (solves >= p.max_lcp_iters) break;
    rebuild_plist(S, m);
    ensure_columns(d, S, m, ld, eps_w, W);
    ++solves;
    if (!solve_on_set(d, S, m, W)) { fail = true; break; }
    int nneg = 0;
    for (int a = tid; a < S.np; a += nt) {
      const int i = S.plist[a];
      if (!(S.z[i] > 0.0)) { S.inP[i] = 0; ++nneg; }
    }
    nneg = block_sum_int(nneg, S.ired);
    if (nneg == 0) {
      for (int i = tid; i < m; i += nt) S.y[i] = S.z[i];
      break;
    }
  }
  // ---- main loop
  while (!fail && solves < p.max_lcp_iters) {
    rebuild_plist(S, m);
    // w = W y + q outside P (over the active columns); most negative entry
    double best = 1.0e300;
    int bi = 0x7fffffff;
    for (int i = tid; i < m; i += nt) {
      if (S.inP[i]) continue;
      double s = S.q[i];
      for (int a = 0; a < S.np; ++a) {
        const int j = S.plist[a];
        s = fma(W[(size_t)i * m + j], S.y[j], s);
      }
      if (s < -tol_w && (s < best || (s == best && i < bi))) { best = s; bi = i; }
    }
    block_argmin(best, bi, S.red, S.ired);
    if (bi == 0x7fffffff) { done = true; break; }
    if (tid == 0) S.inP[bi] = 1;
    // inner loop: restore y_P > 0
    for (;;) {
      if (solves >= p.max_lcp_iters) break;
      rebuild_plist(S, m);
      ensure_columns(d, S, m, ld, eps_w, W);
      ++solves;
      if (!solve_on_set(d, S, m, W)) { fail = true; break; }
      // alpha = min over P with z_i <= 0 of y_i / (y_i - z_i)
      double amin = 1.0e300;
      int dummy = 0;
      for (int a = tid; a < S.np; a += nt) {
        const int i = S.plist[a];
        if (!(S.z[i] > 0.0)) {
          const double yi = S.y[i], zi = S.z[i];
          amin = fmin(amin, (yi - zi) > 0.0 ? yi / (yi - zi) : 0.0);
        }
      }
      block_argmin(amin, dummy, S.red, S.ired);
      if (amin >= 1.0e300) {
        for (int i = tid; i < m; i += nt) S.y[i] = S.z[i];
        break;
      }
      double ymax = 0.0;
      for (int a = tid; a < S.np; a += nt) {
        const int i = S.plist[a];
        const double v = S.y[i] + amin * (S.z[i] - S.y[i]);
        S.y[i] = v;
        ymax = fmax(ymax, v);
      }
      ymax = block_max(ymax, S.red);
      const double tol_y = p.lcp_tol * fmax(ymax, 1e-300);
      for (int a = tid; a < S.np; a += nt) {
        const int i = S.plist[a];
        if (S.y[i] <= tol_y) { S.inP[i] = 0; S.y[i] = 0.0; }
      }
    }
  }
  __syncthreads();
  // ---- results: multipliers (by row), active flags for the next iteration, active slots; and how
  // many rows active now were active in the previous iteration (same active set: all of them)
  __shared__ int s_kept;
  if (tid == 0) s_kept = 0;
  __syncthreads();
  for (int i = tid; i < m; i += nt) {
    const bool a = S.inP[i] && S.y[i] > 0.0;
    const int row = d.wrow[i];
    const int fl = d.init_flag[row];
    if (a && fl >= 0 && (fl & RF_ACTIVE)) atomicAdd(&s_kept, 1);
    d.y[row] = a ? S.y[i] : 0.0;
    d.p_flag[row] = (d.p_flag[row] & RF_STICKY) | RF_WORKING | (a ? RF_ACTIVE : 0);
  }
  __syncthreads();
  if (tid < 32) {                     // active slots in increasing order (ballot compaction)
    int na = 0;
    for (int i0 = 0; i0 < m; i0 += 32) {
      const int i = i0 + tid;
      const bool a = i < m && S.inP[i] && S.y[i] > 0.0;
      const unsigned mk = __ballot_sync(0xffffffffu, a);
      if (a) d.plist[na + __popc(mk & ((1u << tid) - 1u))] = i;
      na += __popc(mk);
    }
    if (tid == 0) {
      ctl->lcp_pivots += solves;
      ctl->admm_iters += admm_it;
      if (fail) atomicCAS(&ctl->status, 0, ST_NOT_SPD);
      else if (!done) atomicCAS(&ctl->status, 0, ST_TIMEOUT);
      ctl->n_active = na;
      ctl->same_active = (s_kept == na && na == ctl->n_active_prev) ? 1 : 0;
    }
  }
}

__global__ void __launch_bounds__(kLcpThreads) contact_kernel(Params p, Dev d) {
  pdl_enter();
  contact_body(p, d);
}

__global__ void __launch_bounds__(kLcpThreads) contact_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan) {
  for_units(tab, plan, PH_CONTACT, [](const Inst& in, int, int) { contact_body(in.p, in.d); });
}

}  // namespace accfem
