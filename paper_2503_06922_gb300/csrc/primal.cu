// OSQP's ADMM on the primal QP of Eq. 23 (the paper's solver, Sec. III.B): min 1/2 dx^T K dx + g^T dx
// subject to A dx <= b over every constraint row (node rows: n^T du_node <= gap).  With the step
// sizes sigma = 1e-6, rho = 0.1 max diag K and relaxation alpha = 1.6, one iteration is
//   xt = (K + sigma I + rho A^T A)^-1 (sigma x - g + A^T (rho z - lam)),  zt = A xt
//   x <- alpha xt + (1 - alpha) x,  zh = alpha zt + (1 - alpha) z
//   z <- min(zh + lam / rho, b),    lam <- lam + rho (zh - z)
// stopped when |A x - z| <= 1e-3 max(|A x|, |z|) and |K x + g + A^T lam| <= 1e-3 max(|K x|, |A^T lam|,
// |g|) (infinity norms, every 10 iterations), as the oracle's lcp.primal_admm; at each test rho adapts
// as in OSQP (rho sqrt(relative primal / relative dual residual), taken when it changes rho by more
// than a factor 5, with a refactorization).  A node row adds
// rho n n^T to its node's translational block, so K + sigma I + rho A^T A keeps K's block-tridiagonal
// form: it is factored once per Newton iteration by a block cyclic reduction and every iteration is
// one 1-column solve with that factor.  The rows with lam > 0 (their bound binds) are the guess that
// starts the exact contact-space active-set method (contact.cu), which gives the unique solution.
//
// One CTA of 1024 threads runs the whole ADMM of a handle: 16 groups of 64 threads take the 6x6
// block work of one node each, and block barriers separate the levels of the reduction and the steps
// of an iteration.  It is launched after the assembly (D, U, g and the rows are final) and before
// the reduction kernels, which overwrite D.
#include "batch.cuh"

namespace accfem {

constexpr int kPrimalThreads = 1024;
constexpr int kPrimalGroups = kPrimalThreads / 64;

// Reduction storage: at the level s where node j is eliminated, pP = its pivot block inverse,
// pEL = K_{j-s, j} and pER = K_{j, j+s}; pD / pE hold the blocks of the current level
// (pE_i = K_{i, i+s}).
__device__ __forceinline__ double* blk(double* base, int node) { return base + (size_t)node * 36; }

// 6x6 Gauss-Jordan inverse of a group's matrix in shared memory (lanes 0..35 own an entry); every
// thread of the CTA calls it (the groups step together).  Returns false if a pivot of an active
// group is not positive (recorded in *bad).
__device__ void group_inverse6(double* A, bool active, int lane, int* bad) {
  const int r = lane / 6, c = lane % 6;
  for (int k = 0; k < 6; ++k) {
    __syncthreads();
    const double akk = A[k * 6 + k];
    double v = 0.0;
    if (active && lane < 36) {
      if (!(akk > 0.0)) {
        if (lane == 0) atomicExch(bad, 1);
      } else {
        const double pk = __drcp_rn(akk);
        const double aij = A[r * 6 + c], aik = A[r * 6 + k], akj = A[k * 6 + c];
        if (r == k && c == k) v = pk;
        else if (r == k) v = akj * pk;
        else if (c == k) v = -aik * pk;
        else v = aij - aik * akj * pk;
      }
    }
    __syncthreads();
    if (active && lane < 36) A[r * 6 + c] = v;
  }
  __syncthreads();
}

__device__ __forceinline__ double block_max_1024(double v, double* s_red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if (lane == 0) s_red[w] = v;
  __syncthreads();
  if (w == 0) {
    double x = s_red[lane];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xffffffffu, x, o));
    if (lane == 0) s_red[32] = x;
  }
  __syncthreads();
  return s_red[32];
}

// Factor of K + sigma I + rho A^T A (in pD / pE on entry) by block cyclic reduction.
__device__ bool primal_factor(const Dev& d, int nf, double (*sM)[6 * 36], int* s_bad) {
  const int g = threadIdx.x >> 6, lane = threadIdx.x & 63;
  int s = 1;
  for (; s < nf; s *= 2) {
    // eliminated nodes j = s, 3s, 5s, ... : pP_j = D_j^-1, pEL_j = E_{j-s}, pER_j = E_j
    const int ne = (nf - s - 1) / (2 * s) + 1;
    for (int r0 = 0; r0 < ne; r0 += kPrimalGroups) {
      const int q = r0 + g;
      const bool act = q < ne;
      const int j = s + 2 * s * q;
      if (act && lane < 36) sM[g][lane] = blk(d.pa_D, j)[lane];
      group_inverse6(sM[g], act, lane, s_bad);
      if (act && lane < 36) {
        blk(d.pa_P, j)[lane] = sM[g][lane];
        blk(d.pa_EL, j)[lane] = blk(d.pa_E, j - s)[lane];
        blk(d.pa_ER, j)[lane] = j + s < nf ? blk(d.pa_E, j)[lane] : 0.0;
      }
    }
    __syncthreads();
    if (*s_bad) return false;
    // kept nodes i = 0, 2s, 4s, ... : D_i -= ER_{i-s}^T P_{i-s} ER_{i-s} + EL_{i+s} P_{i+s} EL_{i+s}^T,
    // E_i <- -EL_{i+s} P_{i+s} ER_{i+s}
    const int nk = (nf - 1) / (2 * s) + 1;
    for (int r0 = 0; r0 < nk; r0 += kPrimalGroups) {
      const int q = r0 + g;
      const int i = 2 * s * q;
      const bool act = q < nk;
      const bool hl = act && i - s >= 0, hr = act && i + s < nf;
      double* T1 = sM[g];            // P_{i-s} ER_{i-s}
      double* T2 = sM[g] + 36;       // P_{i+s} EL_{i+s}^T
      double* T3 = sM[g] + 72;       // P_{i+s} ER_{i+s}
      const int rr = lane / 6, cc = lane % 6;
      if (lane < 36) {
        double t1 = 0.0, t2 = 0.0, t3 = 0.0;
        if (hl) {
          const double* Pl = blk(d.pa_P, i - s);
          const double* Xl = blk(d.pa_ER, i - s);
          for (int k = 0; k < 6; ++k) t1 = fma(Pl[rr * 6 + k], Xl[k * 6 + cc], t1);
        }
        if (hr) {
          const double* Pr = blk(d.pa_P, i + s);
          const double* Lr = blk(d.pa_EL, i + s);
          const double* Rr = blk(d.pa_ER, i + s);
          for (int k = 0; k < 6; ++k) {
            t2 = fma(Pr[rr * 6 + k], Lr[cc * 6 + k], t2);
            t3 = fma(Pr[rr * 6 + k], Rr[k * 6 + cc], t3);
          }
        }
        T1[lane] = t1; T2[lane] = t2; T3[lane] = t3;
      }
      __syncthreads();
      if (act && lane < 36) {
        double dd = blk(d.pa_D, i)[lane], e = 0.0;
        if (hl) {
          const double* Xl = blk(d.pa_ER, i - s);
          for (int k = 0; k < 6; ++k) dd = fma(-Xl[k * 6 + rr], T1[k * 6 + cc], dd);
        }
        if (hr) {
          const double* Lr = blk(d.pa_EL, i + s);
          for (int k = 0; k < 6; ++k) {
            dd = fma(-Lr[rr * 6 + k], T2[k * 6 + cc], dd);
            e = fma(-Lr[rr * 6 + k], T3[k * 6 + cc], e);
          }
        }
        blk(d.pa_D, i)[lane] = dd;
        blk(d.pa_E, i)[lane] = e;
      }
      __syncthreads();
    }
  }
  // the root: node 0
  if (g == 0 && lane < 36) sM[0][lane] = blk(d.pa_D, 0)[lane];
  group_inverse6(sM[0], g == 0, lane, s_bad);
  if (g == 0 && lane < 36) blk(d.pa_P, 0)[lane] = sM[0][lane];
  __syncthreads();
  return *s_bad == 0;
}

// x = (K + sigma I + rho A^T A)^-1 w with the factor (w is overwritten; v is scratch).
__device__ void primal_solve(const Dev& d, int nf, double* w, double* v, double* x) {
  const int tid = threadIdx.x, nt = blockDim.x;
  int smax = 1;
  while (smax * 2 < nf) smax *= 2;
  for (int s = 1; s < nf; s *= 2) {
    const int ne = (nf - s - 1) / (2 * s) + 1;
    for (int t = tid; t < ne * 6; t += nt) {                    // v_j = P_j w_j
      const int j = s + 2 * s * (t / 6), c = t % 6;
      const double* P = blk(d.pa_P, j);
      double a = 0.0;
      for (int k = 0; k < 6; ++k) a = fma(P[c * 6 + k], w[j * 6 + k], a);
      v[j * 6 + c] = a;
    }
    __syncthreads();
    const int nk = (nf - 1) / (2 * s) + 1;
    for (int t = tid; t < nk * 6; t += nt) {                    // w_i -= ER_{i-s}^T v_{i-s} + EL_{i+s} v_{i+s}
      const int i = 2 * s * (t / 6), c = t % 6;
      double a = w[i * 6 + c];
      if (i - s >= 0) {
        const double* X = blk(d.pa_ER, i - s);
        for (int k = 0; k < 6; ++k) a = fma(-X[k * 6 + c], v[(i - s) * 6 + k], a);
      }
      if (i + s < nf) {
        const double* L = blk(d.pa_EL, i + s);
        for (int k = 0; k < 6; ++k) a = fma(-L[c * 6 + k], v[(i + s) * 6 + k], a);
      }
      w[i * 6 + c] = a;
    }
    __syncthreads();
  }
  for (int c = tid; c < 6; c += nt) {                           // the root
    const double* P = blk(d.pa_P, 0);
    double a = 0.0;
    for (int k = 0; k < 6; ++k) a = fma(P[c * 6 + k], w[k], a);
    x[c] = a;
  }
  __syncthreads();
  for (int s = (nf > 1 ? smax : 0); s >= 1; s /= 2) {           // x_j = P_j (w_j - EL_j^T x_{j-s} - ER_j x_{j+s})
    const int ne = (nf - s - 1) / (2 * s) + 1;
    for (int t = tid; t < ne * 6; t += nt) {
      const int j = s + 2 * s * (t / 6), c = t % 6;
      const double* L = blk(d.pa_EL, j);
      const double* R = blk(d.pa_ER, j);
      double a = w[j * 6 + c];
      for (int k = 0; k < 6; ++k) a = fma(-L[k * 6 + c], x[(j - s) * 6 + k], a);
      if (j + s < nf)
        for (int k = 0; k < 6; ++k) a = fma(-R[c * 6 + k], x[(j + s) * 6 + k], a);
      v[j * 6 + c] = a;
    }
    __syncthreads();
    for (int t = tid; t < ne * 6; t += nt) {
      const int j = s + 2 * s * (t / 6), c = t % 6;
      const double* P = blk(d.pa_P, j);
      double a = 0.0;
      for (int k = 0; k < 6; ++k) a = fma(P[c * 6 + k], v[j * 6 + k], a);
      x[j * 6 + c] = a;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kPrimalThreads, 1) primal_admm_kernel(Params p, Dev d) {
  __shared__ double sM[kPrimalGroups][6 * 36];
  __shared__ double s_red[33];
  __shared__ int s_bad;
  pdl_enter();
  Ctl* ctl = d.ctl;
  if (ctl->status != 0 || ctl->converged) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nf = ctl->nf, m = ctl->m;
  if (m == 0) return;                        // no rows: the active-set method starts empty anyway
  if (tid == 0) s_bad = 0;
  // rho = 0.1 max diag K; pD = D + sigma I + rho sum_rows n n^T, pE = U
  double dmax = 0.0;
  for (int t = tid; t < nf * 6; t += nt) dmax = fmax(dmax, d.D[(size_t)(t / 6) * 36 + (t % 6) * 7]);
  dmax = block_max_1024(dmax, s_red);
  const double sigma = 1.0e-6, alpha = 1.6, eps_rel = 1.0e-3;
  double rho = 0.1 * dmax;
  // K + sigma I + rho A^T A from the assembled blocks, factored (again whenever rho changes)
  auto factor = [&]() -> bool {
    for (int t = tid; t < nf * 36; t += nt) {
      const int f = t / 36, e = t % 36, r = e / 6, c = e % 6;
      double v = d.D[t] + (r == c ? sigma : 0.0);
      if (r < 3 && c < 3)
        for (int row = d.c_first[f]; row < d.c_first[f + 1]; ++row)
          v = fma(rho * d.c_w1[3 * row + r], d.c_w1[3 * row + c], v);
      d.pa_D[t] = v;
      d.pa_E[t] = d.U[t];
    }
    __syncthreads();
    return primal_factor(d, nf, sM, &s_bad);
  };
  if (!factor()) {
    if (tid == 0) atomicCAS(&ctl->status, 0, ST_NOT_SPD);
    return;
  }
  for (int t = tid; t < nf * 6; t += nt) d.pa_x[t] = 0.0;
  for (int r = tid; r < m; r += nt) { d.pa_z[r] = 0.0; d.pa_lam[r] = 0.0; }
  __syncthreads();
  int it = 0;
  while (it < p.admm_iters) {
    ++it;
    // right-hand side sigma x - g + A^T (rho z - lam)
    for (int t = tid; t < nf * 6; t += nt) {
      const int f = t / 6, c = t % 6;
      double v = fma(sigma, d.pa_x[t], -d.g[t]);
      if (c < 3)
        for (int row = d.c_first[f]; row < d.c_first[f + 1]; ++row)
          v = fma(d.c_w1[3 * row + c], fma(rho, d.pa_z[row], -d.pa_lam[row]), v);
      d.pa_w[t] = v;
    }
    __syncthreads();
    primal_solve(d, nf, d.pa_w, d.pa_v, d.pa_xt);
    // relaxation, projection on z <= b, multiplier update (rows by their node)
    for (int r = tid; r < m; r += nt) {
      const int f = d.c_node[r];
      const double* n = d.c_w1 + 3 * r;
      const double zt = fma(n[0], d.pa_xt[f * 6], fma(n[1], d.pa_xt[f * 6 + 1], n[2] * d.pa_xt[f * 6 + 2]));
      const double zh = fma(alpha, zt, (1.0 - alpha) * d.pa_z[r]);
      const double zn = fmin(zh + d.pa_lam[r] / rho, d.c_gap[r]);
      d.pa_lam[r] = fma(rho, zh - zn, d.pa_lam[r]);
      d.pa_z[r] = zn;
    }
    for (int t = tid; t < nf * 6; t += nt) d.pa_x[t] = fma(alpha, d.pa_xt[t], (1.0 - alpha) * d.pa_x[t]);
    __syncthreads();
    if (it % 10 == 0) {
      // residuals: |A x - z| against max(|A x|, |z|); |K x + g + A^T lam| against max(|K x|, |A^T lam|, |g|)
      double rp = 0.0, ax = 0.0, zm = 0.0;
      for (int r = tid; r < m; r += nt) {
        const int f = d.c_node[r];
        const double* n = d.c_w1 + 3 * r;
        const double a = fma(n[0], d.pa_x[f * 6], fma(n[1], d.pa_x[f * 6 + 1], n[2] * d.pa_x[f * 6 + 2]));
        rp = fmax(rp, fabs(a - d.pa_z[r]));
        ax = fmax(ax, fabs(a));
        zm = fmax(zm, fabs(d.pa_z[r]));
      }
      double rd = 0.0, kx = 0.0, al = 0.0, gm = 0.0;
      for (int t = tid; t < nf * 6; t += nt) {
        const int f = t / 6, c = t % 6;
        double k = 0.0;
        for (int q = 0; q < 6; ++q) k = fma(d.D[(size_t)f * 36 + c * 6 + q], d.pa_x[f * 6 + q], k);
        if (f + 1 < nf)
          for (int q = 0; q < 6; ++q) k = fma(d.U[(size_t)f * 36 + c * 6 + q], d.pa_x[(f + 1) * 6 + q], k);
        if (f > 0)
          for (int q = 0; q < 6; ++q) k = fma(d.U[(size_t)(f - 1) * 36 + q * 6 + c], d.pa_x[(f - 1) * 6 + q], k);
        double a = 0.0;
        if (c < 3)
          for (int row = d.c_first[f]; row < d.c_first[f + 1]; ++row) a = fma(d.c_w1[3 * row + c], d.pa_lam[row], a);
        rd = fmax(rd, fabs(k + d.g[t] + a));
        kx = fmax(kx, fabs(k));
        al = fmax(al, fabs(a));
        gm = fmax(gm, fabs(d.g[t]));
      }
      rp = block_max_1024(rp, s_red);
      ax = block_max_1024(ax, s_red);
      zm = block_max_1024(zm, s_red);
      rd = block_max_1024(rd, s_red);
      kx = block_max_1024(kx, s_red);
      al = block_max_1024(al, s_red);
      gm = block_max_1024(gm, s_red);
      const double sp = fmax(ax, zm), sd = fmax(fmax(kx, al), gm);
      if (rp <= eps_rel * sp && rd <= eps_rel * sd) break;
      // OSQP's adaptive step size: rho scaled by sqrt(relative primal / relative dual residual) when
      // that changes it by more than a factor 5, and the matrix refactored
      if (rp > 0.0 && rd > 0.0 && sp > 0.0 && sd > 0.0) {
        const double rn = rho * sqrt((rp / sp) / (rd / sd));
        if (rn > 5.0 * rho || rn < 0.2 * rho) {
          rho = rn;
          if (!factor()) {
            if (tid == 0) atomicCAS(&ctl->status, 0, ST_NOT_SPD);
            return;
          }
        }
      }
    }
  }
  // the guess of the active rows: the bound binds (lam > 0)
  for (int r = tid; r < m; r += nt) d.pa_guess[r] = d.pa_lam[r] > 0.0 ? 1 : 0;
  if (tid == 0) ctl->admm_iters += it;
}

}  // namespace accfem
