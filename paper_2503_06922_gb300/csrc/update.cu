// Newton update with the step limiter (Eq. 25-27), convergence test, and the start pose of a
// solve (prescribed feed, Eq. 14-15; warm start from the resident pose).
#include "batch.cuh"

namespace accfem {

// dx = dx_free - X y over the active working-set slots; per-node maxima of |du|,
// max(|du|, r_o |dtheta|) and of the residual g + A^T y.  Block: 32 nodes x 6 components.
__device__ __forceinline__ void step_body(const Params& p, const Dev& d, int bx) {
  __shared__ double s_dx[32][6];
  __shared__ double s_r[32][6];
  __shared__ int s_j[kMaxWorking];            // active working-set slots and their multipliers
  __shared__ double s_y[kMaxWorking];
  __shared__ double s_aac[kAccelDepth][32][3];  // translations of the step differences c_j
  __shared__ double s_aap[6][kAccelParts];      // least-squares sums per component warp
  Ctl* ctl = d.ctl;
  if (ctl->status != 0 || ctl->converged) return;
  const int nf = ctl->nf;
  const int fl = threadIdx.x, c = threadIdx.y;
  const int f = bx * 32 + fl;
  const bool act = f < nf;
  const size_t ld = p.nrhs_cap;
  const int na = ctl->n_active;
  for (int a = threadIdx.y * 32 + threadIdx.x; a < na; a += 192) {
    const int j = d.plist[a];
    s_j[a] = j;
    s_y[a] = d.y[d.wrow[j]];
  }
  __syncthreads();
  if (act) {
    double v = d.B[((size_t)f * 6 + c) * ld];
    const double* bx_col = d.B + ((size_t)f * 6 + c) * ld + 1;
    for (int a = 0; a < na; ++a) v = fma(-bx_col[s_j[a]], s_y[a], v);
    s_dx[fl][c] = v;
    d.dx[(size_t)f * 6 + c] = v;
    double r = d.g[(size_t)f * 6 + c];
    if (c < 3) {
      for (int row = d.c_first[f]; row < d.c_first[f + 1]; ++row) r = fma(d.c_w1[3 * row + c], d.y[row], r);
      if (p.contact_model == kContactSegment && f + 1 < nf)   // segment rows of the next element weigh this node too
        for (int row = d.c_first[f + 1]; row < d.c_first[f + 2]; ++row)
          if (d.c_node2[row] == f) r = fma(d.c_w2[3 * row + c], d.y[row], r);
    }
    s_r[fl][c] = fabs(r);
  }
  __syncthreads();
  double rr_node = 0.0;
  if (act && c == 0)
    rr_node = fmax(fmax(fmax(s_r[fl][0], s_r[fl][1]), fmax(s_r[fl][2], s_r[fl][3])), fmax(s_r[fl][4], s_r[fl][5]));
  // Anderson acceleration: differences c_j = f_{k-j+1} - f_{k-j} of this step and the held ones,
  // least-squares sums (weight 1 on translations, r_o^2 on rotations) and their nodal translations
  {
    const int n_h = ctl->aa_n, k_it = ctl->iter;
    double cj[kAccelDepth] = {0.0, 0.0, 0.0};
    if (act) {
      double prev = s_dx[fl][c];
      for (int j = 1; j <= n_h; ++j) {
        const double h = d.aa_f[((size_t)((k_it - j) % kAccelSlots) * p.M + f) * 6 + c];
        cj[j - 1] = prev - h;
        prev = h;
      }
      if (c < 3)
        for (int j = 0; j < kAccelDepth; ++j) s_aac[j][fl][c] = cj[j];
    }
    const double wv = c < 3 ? 1.0 : p.r_o * p.r_o;
    const double fk = act ? s_dx[fl][c] : 0.0;
    double part[kAccelParts] = {wv * cj[0] * cj[0], wv * cj[0] * cj[1], wv * cj[0] * cj[2], wv * cj[1] * cj[1],
                                wv * cj[1] * cj[2], wv * cj[2] * cj[2], wv * cj[0] * fk, wv * cj[1] * fk, wv * cj[2] * fk,
                                c < 3 ? fk * fk : 0.0};
#pragma unroll
    for (int i = 0; i < kAccelParts; ++i) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part[i] += __shfl_xor_sync(0xffffffffu, part[i], o);
    }
    if (threadIdx.x == 0)
#pragma unroll
      for (int i = 0; i < kAccelParts; ++i) s_aap[c][i] = part[i];
  }
  __syncthreads();
  if (threadIdx.y == 0 && threadIdx.x < kAccelParts) {
    double v = 0.0;
    for (int w = 0; w < 6; ++w) v += s_aap[w][threadIdx.x];
    d.aa_part[(size_t)bx * kAccelParts + threadIdx.x] = v;
  }
  if (act && c == 0)
    for (int j = 0; j < ctl->aa_n; ++j) {
      const double n2 = fma(s_aac[j][fl][0], s_aac[j][fl][0], fma(s_aac[j][fl][1], s_aac[j][fl][1], s_aac[j][fl][2] * s_aac[j][fl][2]));
      atomicMax(&ctl->aa_cmax_bits[j], dbits(sqrt(n2)));
    }
  __syncthreads();
  if (act && c < 3) {
    // reversal test of the limiter: this step against the previous one (translations)
    s_r[fl][c] = s_dx[fl][c] * d.du_prev[(size_t)f * 3 + c];
    d.du_prev[(size_t)f * 3 + c] = s_dx[fl][c];
  }
  __syncthreads();
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    double rev = 0.0;
    for (int k = 0; k < 32 && bx * 32 + k < nf; ++k) rev += s_r[k][0] + s_r[k][1] + s_r[k][2];
    d.rev_part[bx] = rev;
  }
  if (act && c == 0) {
    double du = sqrt(s_dx[fl][0] * s_dx[fl][0] + s_dx[fl][1] * s_dx[fl][1] + s_dx[fl][2] * s_dx[fl][2]);
    double dt = sqrt(s_dx[fl][3] * s_dx[fl][3] + s_dx[fl][4] * s_dx[fl][4] + s_dx[fl][5] * s_dx[fl][5]);
    double st = fmax(du, p.r_o * dt);
    atomicMax(&ctl->umax_bits, dbits(du));
    atomicMax(&ctl->step_bits, dbits(st));
    atomicMax(&ctl->res_bits, dbits(rr_node));
  }
}

__global__ void __launch_bounds__(192) step_kernel(Params p, Dev d) {
  pdl_enter();
  step_body(p, d, blockIdx.x);
}

__global__ void __launch_bounds__(192) step_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan) {
  for_units(tab, plan, PH_STEP, [](const Inst& in, int bx, int) { step_body(in.p, in.d, bx); });
}

// Step limiter (Eq. 25-27 with an adaptive bound): alpha = min(1, rho / max |du|).  A step that
// points against the previous one (sum_i du_i . du_i^prev < 0, summed over the step blocks in a
// fixed order) is an overshoot, unless the previous step was an accelerated one: rho drops to half of
// min(rho, max |du|), so the step is at most halved and a repeating cycle shrinks geometrically;
// otherwise rho grows by 1.5 back towards beta0.
// Anderson acceleration (depth kAccelDepth) of the iteration x <- x (+) f(x), f the unscaled Newton
// step, in the first kAccelIters iterations of a solve with the FP64 tangent: while the active rows (by
// node and triangle) stay those of the previous iteration and the step is not clipped ("steady"; rows
// that enter or leave the detection without becoming active do not change the step), gamma minimises |W (f_k - sum_j gamma_j c_j)| over the n held
// differences c_j = f_{k-j+1} - f_{k-j} (W: weight r_o on rotations; a relative ridge 1e-10 max G_jj),
// and the increment f_k - sum_j gamma_j (d_{k-j} + c_j), d_{k-j} the increment applied at iterate k-j,
// is taken when sum |gamma_j| <= kAccelGammaMax and a bound on its largest nodal translation,
// max|f_k| + sum_j |gamma_j| (max|d_{k-j}| + max|c_j|), stays within beta0 (the step limit that keeps
// a node from crossing an undetected wall; the adaptive rho only damps overshoots, which the
// extrapolation itself removes).  The block's threads reduce
// the per-step-block partial sums; thread 0 evaluates the rule.
struct LimOut {
  double rho, alpha, bound, nrm2, gamma[kAccelDepth];
  int accel, steady;
};

__device__ void limiter_block(const Params& p, const Dev& d, const Ctl* ctl, LimOut* out) {
  __shared__ double s_red[kAccelParts + 1][4];
  const int nb = (ctl->nf + 31) / 32;
  const int tid = threadIdx.x + threadIdx.y * blockDim.x, nthr = blockDim.x * blockDim.y;
  const int lane = tid & 31, w = tid >> 5;
  double acc[kAccelParts + 1];
#pragma unroll
  for (int i = 0; i <= kAccelParts; ++i) acc[i] = 0.0;
  for (int b = tid; b < nb; b += nthr) {
    acc[0] += d.rev_part[b];
#pragma unroll
    for (int i = 0; i < kAccelParts; ++i) acc[i + 1] += d.aa_part[(size_t)b * kAccelParts + i];
  }
  // Threads from `live` on hold +0.0.  The butterfly rounds whose partners all hold +0.0 (o >= live)
  // and the sums of the warps without data are left out: adding +0.0 changes no bit of a total that
  // starts from +0.0, and each left-out addition costs the SMSP's FP64 pipe 64 cycles.
  const int live = min(nb, nthr);
#pragma unroll
  for (int i = 0; i <= kAccelParts; ++i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      if (o < live) acc[i] += __shfl_xor_sync(0xffffffffu, acc[i], o);
  }
  if (lane == 0 && w < 4)
#pragma unroll
    for (int i = 0; i <= kAccelParts; ++i) s_red[i][w] = acc[i];
  __syncthreads();
  if (tid == 0) {
    const int nw = min(min((nthr + 31) / 32, 4), (live + 31) / 32);
    double S[kAccelParts + 1];
    for (int i = 0; i <= kAccelParts; ++i) {
      S[i] = 0.0;
      for (int k = 0; k < nw; ++k) S[i] += s_red[i][k];
    }
    const double rev = S[0];
    double rho = ctl->rho;
    const double umax = __longlong_as_double((long long)ctl->umax_bits);
    const bool reverse = ctl->has_prev && rev < 0.0 && !ctl->aa_prev;
    if (ctl->has_prev) {
      if (reverse) rho = fmax(0.5 * fmin(rho, umax), p.beta0 * 9.094947017729282e-13);   // beta0 / 2^40
      else rho = fmin(1.5 * rho, p.beta0);
    }
    double a = umax <= rho ? 1.0 : rho / umax;
    const int n = ctl->aa_n;
    // Anderson steps only in the first kAccelIters iterations and with the FP64 tangent (the FP32
    // tangent's error in the soft modes is of order one, so its successive steps are not samples of
    // one smooth map)
    const bool anderson = ctl->iter < kAccelIters && !(p.precision == kPrecisionMixed && !ctl->fp64_tangent);
    out->steady = (ctl->has_prev && a == 1.0 && ctl->same_active && anderson) ? 1 : 0;
    out->accel = 0;
    out->bound = 0.0;
    // otherwise the secant over-relaxation of a slow monotone mode: after a full step, an unclipped step
    // with the same constraint rows, pointing the same way as the previous one (cosine >= 0.99) and
    // shrinking by lam = |du| / |du_prev| in [0.5, 0.98], is extended to alpha = min(1 / (1 - lam), 8, rho / max|du|)
    const double nrm2 = S[10];
    if (!anderson && ctl->has_prev && !reverse && ctl->alpha == 1.0 && a == 1.0 && ctl->same_set &&
        ctl->nrm2_prev > 0.0 && nrm2 > 0.0) {
      const double lam = sqrt(nrm2 / ctl->nrm2_prev);
      const double cosang = rev / sqrt(nrm2 * ctl->nrm2_prev);
      if (cosang >= 0.99 && lam >= 0.5 && lam <= 0.98) a = fmin(fmin(1.0 / (1.0 - lam), 8.0), rho / umax);
    }
    out->nrm2 = nrm2;
    for (int j = 0; j < kAccelDepth; ++j) out->gamma[j] = 0.0;
    if (out->steady && n >= 1) {
      // normal equations (G + ridge) gamma = b, n <= 3, by Gaussian elimination (G symmetric positive)
      double G[3][3] = {{S[1], S[2], S[3]}, {S[2], S[4], S[5]}, {S[3], S[5], S[6]}};
      double bv[3] = {S[7], S[8], S[9]};
      double dmx = 0.0;
      for (int j = 0; j < n; ++j) dmx = fmax(dmx, G[j][j]);
      for (int j = 0; j < n; ++j) G[j][j] += 1e-10 * dmx;
      bool ok = dmx > 0.0;
      for (int c = 0; c < n && ok; ++c) {
        if (!(G[c][c] > 0.0)) { ok = false; break; }
        for (int r = c + 1; r < n; ++r) {
          const double fct = G[r][c] / G[c][c];
          for (int q = c; q < n; ++q) G[r][q] = fma(-fct, G[c][q], G[r][q]);
          bv[r] = fma(-fct, bv[c], bv[r]);
        }
      }
      double gam[3] = {0.0, 0.0, 0.0};
      if (ok)
        for (int c = n - 1; c >= 0; --c) {
          double v = bv[c];
          for (int q = c + 1; q < n; ++q) v = fma(-G[c][q], gam[q], v);
          gam[c] = v / G[c][c];
        }
      double gsum = 0.0;
      for (int j = 0; j < n; ++j) gsum += fabs(gam[j]);
      if (ok && isfinite(gsum) && gsum <= kAccelGammaMax) {
        double bound = umax;
        for (int j = 1; j <= n; ++j)
          bound = fma(fabs(gam[j - 1]),
                      ctl->aa_dmax[(ctl->iter - j) % kAccelDepth] + __longlong_as_double((long long)ctl->aa_cmax_bits[j - 1]),
                      bound);
        if (bound <= p.beta0) {
          out->accel = 1;
          out->bound = bound;
          for (int j = 0; j < n; ++j) out->gamma[j] = gam[j];
        }
      }
    }
    out->rho = rho;
    out->alpha = a;
  }
  __syncthreads();
}

// x <- x + alpha du, T <- exp([alpha dtheta]x) T.  Every row of the node outside the working set is
// checked against the applied step: w = b - alpha n . du < -tol marks it violated (it joins the
// working set in the next iteration, and this iteration cannot converge; at convergence alpha = 1).
__device__ __forceinline__ void apply_body(const Params& p, const Dev& d, int bx) {
  __shared__ LimOut s_lim;
  Ctl* ctl = d.ctl;
  if (ctl->status != 0 || ctl->converged) return;
  const int nf = ctl->nf;
  limiter_block(p, d, ctl, &s_lim);
  if (bx == 0 && threadIdx.x == 0) {             // the decision, for the control update
    ctl->lim_rho = s_lim.rho;
    ctl->lim_alpha = s_lim.alpha;
    ctl->lim_bound = s_lim.bound;
    ctl->lim_accel = s_lim.accel;
    ctl->lim_steady = s_lim.steady;
    ctl->lim_nrm2 = s_lim.nrm2;
  }
  const double alpha = s_lim.alpha;
  const int accel = s_lim.accel;
  const int f = bx * 128 + threadIdx.x;
  if (f < nf) {
    const int node = ctl->k + 1 + f;
    const int k_it = ctl->iter, n_h = ctl->aa_n;
    // the increment of free node g: alpha dx, or f_k - sum_j gamma_j (d_{k-j} + f_{k-j+1} - f_{k-j})
    auto increment = [&](int g, double* out) {
      const double* dxg = d.dx + (size_t)g * 6;
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        double v = accel ? dxg[c] : alpha * dxg[c];
        if (accel) {
          double prev = dxg[c];
          for (int j = 1; j <= n_h; ++j) {
            const size_t at = ((size_t)((k_it - j) % kAccelSlots) * p.M + g) * 6 + c;
            const double h = d.aa_f[at];
            v = fma(-s_lim.gamma[j - 1], d.aa_d[at] + (prev - h), v);
            prev = h;
          }
        }
        out[c] = v;
      }
    };
    const double* dx = d.dx + (size_t)f * 6;
    double inc[6];
    increment(f, inc);
    // this iterate joins the held ones (its slot held the oldest, already read above)
    const size_t at = ((size_t)(k_it % kAccelSlots) * p.M + f) * 6;
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      d.aa_f[at + c] = dx[c];
      d.aa_d[at + c] = inc[c];
    }
    for (int row = d.c_first[f]; row < d.c_first[f + 1]; ++row) {
      if (d.rslot[row] >= 0) continue;
      const double* n = d.c_w1 + 3 * row;
      double an = fma(n[0], inc[0], fma(n[1], inc[1], n[2] * inc[2]));
      if (d.c_node2[row] >= 0) {                    // a segment row: the element's near node moves too
        double inc2[6];
        increment(d.c_node2[row], inc2);
        const double* n2 = d.c_w2 + 3 * row;
        an = fma(n2[0], inc2[0], fma(n2[1], inc2[1], fma(n2[2], inc2[2], an)));
      }
      const double w = d.c_gap[row] - an;
      if (w < -p.tol) {
        d.p_flag[row] = RF_VIOLATED;
        ctl->incomplete = 1;
      }
    }
    d.px[node] += inc[0];
    d.py[node] += inc[1];
    d.pz[node] += inc[2];
    double th[3] = {inc[3], inc[4], inc[5]};
    double dq[4], q[4] = {d.qw[node], d.qx[node], d.qy[node], d.qz[node]}, r[4];
    quat_exp(th, dq);
    quat_mul(dq, q, r);
    double in = rsqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
    if (r[0] < 0.0) in = -in;
    d.qw[node] = r[0] * in; d.qx[node] = r[1] * in; d.qy[node] = r[2] * in; d.qz[node] = r[3] * in;
  }
}

__global__ void __launch_bounds__(128) apply_kernel(Params p, Dev d) {
  pdl_enter();
  apply_body(p, d, blockIdx.x);
}

__global__ void __launch_bounds__(128) apply_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan) {
  for_units(tab, plan, PH_APPLY, [](const Inst& in, int bx, int) { apply_body(in.p, in.d, bx); });
}

// End of an iteration (one thread): limiter bookkeeping, iteration count, convergence (unscaled
// step below tol with an unchanged constraint set and no violated row outside the working set, so
// that the working-set LCP solution solves the LCP of all rows), and -- inside the device-side
// Newton graph --
// the loop condition: keep iterating while no error, not converged and fewer than max_iter
// iterations; a separate count of loop passes bounds the loop whatever the other kernels did.
__device__ __forceinline__ void ctl_update(const Params& p, const Dev& d) {
  Ctl* c = d.ctl;
  // mixed precision: a non-positive pivot of the FP32 tangent (its condition number grows like the
  // cube of the element count) switches this solve to the FP64 tangent; the failed iteration
  // applied no step and is repeated
  if (c->status == ST_NOT_SPD && p.precision == kPrecisionMixed && !c->fp64_tangent) {
    // the failed iteration ran no step or apply kernel: it counts, and the held iterates restart
    c->status = 0;
    c->fp64_tangent = 1;
    c->aa_n = 0;
    c->aa_prev = 0;
    c->iter += 1;
  } else if (c->status == 0 && !c->converged) {
    const double step = __longlong_as_double((long long)c->step_bits);
    const double umax = __longlong_as_double((long long)c->umax_bits);
    c->rho = c->lim_rho;
    c->alpha = c->lim_alpha;
    // the held iterates: this one joins them while the iteration is steady, else it alone remains
    c->aa_dmax[c->iter % kAccelDepth] = c->lim_accel ? c->lim_bound : c->lim_alpha * umax;
    c->aa_n = c->lim_steady ? min(c->aa_n + 1, kAccelDepth) : 1;
    c->aa_prev = c->lim_accel;
    c->n_active_prev = c->n_active;
    c->nrm2_prev = c->lim_nrm2;
    c->has_prev = 1;
    c->iter += 1;
    if (step <= p.tol && c->same_set && !c->incomplete) c->converged = 1;
  }
  c->loops += 1;
}

__global__ void ctl_kernel(Params p, Dev d, cudaGraphConditionalHandle h, int max_iter, int set_cond) {
  pdl_enter();
  Ctl* c = d.ctl;
  ctl_update(p, d);
  if (set_cond) {
    unsigned int cont = (c->status == 0 && !c->converged && c->iter < max_iter && c->loops < max_iter) ? 1u : 0u;
    cudaGraphSetConditional(h, cont);
  }
}

// Start pose of a solve.  mode 0: straight on the entrance axis; mode 1: follow the path of the
// previous pose (material point s takes the old pose of material point s + (delta - delta_old):
// linear in x, geodesic in the rotation between nodes, straight along the tip axis beyond the
// old tip); mode 2: poses already uploaded.  Nodes i <= k are then clamped on the axis.
__device__ __forceinline__ void start_body(const Params& p, const Dev& d, int mode, double delta, double delta_old, int k, int i) {
  if (i >= p.N) return;
  const double* dir = p.E0;    // column 0 of E0: (E0[0], E0[3], E0[6])
  double x[3], q[4];
  if (mode == 1) {
    const double s = i * p.l0 + (delta - delta_old);
    if (s >= p.L) {
      const int t = p.M;
      double T[9];
      quat_to_mat(d.ow[t], d.oqx[t], d.oqy[t], d.oqz[t], T);
      double e = s - p.L;
      x[0] = d.ox[t] + e * T[0]; x[1] = d.oy[t] + e * T[3]; x[2] = d.oz[t] + e * T[6];
      q[0] = d.ow[t]; q[1] = d.oqx[t]; q[2] = d.oqy[t]; q[3] = d.oqz[t];
    } else if (s <= 0.0) {
      double T[9];
      quat_to_mat(d.ow[0], d.oqx[0], d.oqy[0], d.oqz[0], T);
      x[0] = d.ox[0] + s * T[0]; x[1] = d.oy[0] + s * T[3]; x[2] = d.oz[0] + s * T[6];
      q[0] = d.ow[0]; q[1] = d.oqx[0]; q[2] = d.oqy[0]; q[3] = d.oqz[0];
    } else {
      int j = (int)floor(s / p.l0);
      if (j > p.M - 1) j = p.M - 1;
      const double f = (s - j * p.l0) / p.l0;
      x[0] = (1.0 - f) * d.ox[j] + f * d.ox[j + 1];
      x[1] = (1.0 - f) * d.oy[j] + f * d.oy[j + 1];
      x[2] = (1.0 - f) * d.oz[j] + f * d.oz[j + 1];
      double qa[4] = {d.ow[j], d.oqx[j], d.oqy[j], d.oqz[j]};
      double qb[4] = {d.ow[j + 1], d.oqx[j + 1], d.oqy[j + 1], d.oqz[j + 1]};
      double qai[4] = {qa[0], -qa[1], -qa[2], -qa[3]}, rel[4], th[3], dq[4];
      quat_mul(qai, qb, rel);               // body-frame relative rotation
      quat_log(rel, th);
      th[0] *= f; th[1] *= f; th[2] *= f;
      quat_exp(th, dq);
      quat_mul(qa, dq, q);
    }
  } else if (mode == 0) {
    double s = (i * p.l0 - p.L) + delta;
    x[0] = p.e[0] + s * dir[0]; x[1] = p.e[1] + s * dir[3]; x[2] = p.e[2] + s * dir[6];
    q[0] = p.q0[0]; q[1] = p.q0[1]; q[2] = p.q0[2]; q[3] = p.q0[3];
  } else {
    x[0] = d.px[i]; x[1] = d.py[i]; x[2] = d.pz[i];
    q[0] = d.qw[i]; q[1] = d.qx[i]; q[2] = d.qy[i]; q[3] = d.qz[i];
  }
  if (i <= k) {
    double s = (i * p.l0 - p.L) + delta;
    x[0] = p.e[0] + s * dir[0]; x[1] = p.e[1] + s * dir[3]; x[2] = p.e[2] + s * dir[6];
    q[0] = p.q0[0]; q[1] = p.q0[1]; q[2] = p.q0[2]; q[3] = p.q0[3];
  }
  double in = rsqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (q[0] < 0.0) in = -in;
  d.px[i] = x[0]; d.py[i] = x[1]; d.pz[i] = x[2];
  d.qw[i] = q[0] * in; d.qx[i] = q[1] * in; d.qy[i] = q[2] * in; d.qz[i] = q[3] * in;
}

__global__ void __launch_bounds__(128) start_kernel(Params p, Dev d, int mode, double delta, double delta_old, int k) {
  start_body(p, d, mode, delta, delta_old, k, blockIdx.x * blockDim.x + threadIdx.x);
}

// Start of the batched solves: block (x, j) sets up begun instance bg[j].member: block 0 copies its
// staged control block; for a warm start the resident pose is saved as the path to follow.
__global__ void __launch_bounds__(128) batch_begin_kernel(const Inst* __restrict__ tab, const Ctl* __restrict__ staged,
                                                          const BatchBegin* __restrict__ bg) {
  const BatchBegin b = bg[blockIdx.y];
  const Dev& d = tab[b.member].d;
  const int n_nodes = tab[b.member].p.N;
  if (blockIdx.x == 0 && threadIdx.x == 0) *d.ctl = staged[blockIdx.y];
  const int i = blockIdx.x * 128 + threadIdx.x;
  if (b.mode == 1 && i < n_nodes) {
    d.ox[i] = d.px[i]; d.oy[i] = d.py[i]; d.oz[i] = d.pz[i];
    d.ow[i] = d.qw[i]; d.oqx[i] = d.qx[i]; d.oqy[i] = d.qy[i]; d.oqz[i] = d.qz[i];
  }
}

__global__ void __launch_bounds__(128) start_batch(const Inst* __restrict__ tab, const BatchBegin* __restrict__ bg) {
  const BatchBegin b = bg[blockIdx.y];
  start_body(tab[b.member].p, tab[b.member].d, b.mode, b.delta, b.delta_old, b.k, blockIdx.x * 128 + threadIdx.x);
}

// End of a batched iteration (one block of 1024 threads, thread i = instance i): the control update
// of every instance in flight (as ctl_kernel when do_ctl), then the plan of the next iteration --
// the instances that keep iterating (no error, not converged, under the iteration cap) and per
// phase the exclusive prefix of their unit counts.  An instance that stops leaves the flight.
// Without do_ctl (start of an advance) it records the iteration budget max_passes; in the batch
// graph it sets the loop condition: some instance iterates and fewer than that many iterations
// were run by this advance.
__global__ void __launch_bounds__(1024) batch_plan_kernel(const Inst* __restrict__ tab, Plan* plan, int n_inst, int do_ctl,
                                                          int max_passes, cudaGraphConditionalHandle h, int set_cond) {
  __shared__ int s_warp[32];
  __shared__ int s_nf[kMaxBatch];
  pdl_enter();
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  int go = 0, nf = 0;
  if (tid < n_inst) {
    const Params& p = tab[tid].p;
    const Dev& d = tab[tid].d;
    Ctl* c = d.ctl;
    if (c->live) {
      if (do_ctl) ctl_update(p, d);
      go = (c->status == 0 && !c->converged && c->iter < p.max_newton && c->loops < p.max_newton) ? 1 : 0;
      if (!go) c->live = 0;
      nf = c->nf;
    }
  }
  int v = go;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  if (lane == 31) s_warp[w] = v;
  __syncthreads();
  if (w == 0) {
    int x = s_warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    s_warp[lane] = x;
  }
  __syncthreads();
  const int pos = v - go + (w > 0 ? s_warp[w - 1] : 0);
  const int n_act = s_warp[31];
  if (go) {
    plan->act[pos] = tid;
    s_nf[pos] = nf;
  }
  __syncthreads();
  for (int ph = w; ph < kPhases; ph += 32) {
    int run = 0;
    if (lane == 0) plan->pre[ph][0] = 0;
    for (int base = 0; base < n_act; base += 32) {
      const int j = base + lane;
      int u = j < n_act ? phase_gx(ph, s_nf[j]) * phase_gy(ph) : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, u, o);
        if (lane >= o) u += t;
      }
      if (j < n_act) plan->pre[ph][j + 1] = run + u;
      run += __shfl_sync(0xffffffffu, u, 31);
    }
  }
  if (tid == 0) {
    plan->n_act = n_act;
    const int passes = do_ctl ? plan->passes + 1 : 0;
    plan->passes = passes;
    if (!do_ctl) plan->max_passes = max_passes;
    if (set_cond) cudaGraphSetConditional(h, (n_act > 0 && passes < plan->max_passes) ? 1u : 0u);
  }
}

}  // namespace accfem
