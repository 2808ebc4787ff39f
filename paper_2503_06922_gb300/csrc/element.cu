// Corotational beam element: internal force and material tangent (Sec. II.B, Eq. 20; the
// element-level parallel update of Sec. III.C).  One warp per element.
//
// Element e joins nodes a = e and b = e + 1.  Rigid frame R_r = [e1 e2 e3]: e1 along the chord,
// e3 normal to e1 and the mean q of the nodal second section axes.  Local deformations
// d_l = [l - l0, log(R_r^T T_a), log(R_r^T T_b)], constant local stiffness K_l (EA/l0, GJ/l0,
// EI/l0 [[4 2][2 4]] per bending plane; each element has its own modulus, Sec. II.A).  With B = dd_l/dd (spatial spins, local components):
//   F = E B^T K_l d_l,   K = E B^T K_l B E^T,   E = blockdiag(R_r, R_r, R_r, R_r).
// Output record (doubles): [0, 78) upper triangle of K row-major, [78, 90) F = [F_a M_a F_b M_b].
#include "batch.cuh"

namespace accfem {

__constant__ unsigned char c_up_i[78];
__constant__ unsigned char c_up_j[78];

// Per-warp scratch for the prelude: every FP64 warp instruction occupies the SMSP's FP64 pipe for
// 64 cycles whatever its lane mask, so independent entries go to different lanes.
struct ElemShared {
  double T[2][9];      // nodal triads a, b (row-major)
  double Rr[9];        // rigid frame, row-major, columns e1 e2 e3
  double Rab[2][9];    // R_r^T T_a, R_r^T T_b
  double th[2][3];     // local rotations
  double Ti[2][9];     // Tsinv(theta_a), Tsinv(theta_b)
  double B[7][12];     // B (local), then B E^T (global comps)
  double H[7][12];     // K_l B E^T
  float B32[7][12];    // mixed precision: B E^T and K_l B E^T in FP32
  float H32[7][12];
};

// Warp body: element k + bx * kWarpsPerElemBlock + wsub (wsub < kWarpsPerElemBlock: the element's
// place in its work unit), computed by one warp with its own scratch S.  kMixed: the tangent products
// H = K_l (B E^T) and K = (B E^T)^T H take FP32 operands and FP32 accumulation; the element force
// (the Newton residual) stays FP64.
template <bool kMixed>
__device__ __forceinline__ void element_warp(const Params& p, const Dev& d, int bx, int wsub, ElemShared& S) {
  const int lane = threadIdx.x & 31;
  const int wib = wsub;
  Ctl* ctl = d.ctl;
  if (bx == 0 && wsub == 0 && lane == 0) {           // reset the per-iteration reductions
    ctl->umax_bits = 0ull; ctl->step_bits = 0ull; ctl->res_bits = 0ull;
#pragma unroll
    for (int j = 0; j < kAccelDepth; ++j) ctl->aa_cmax_bits[j] = 0ull;
    ctl->incomplete = 0;
  }
  const int e = ctl->k + bx * kWarpsPerElemBlock + wib;
  if (e >= p.M || ctl->status != 0 || ctl->converged) return;
  const int a = e, b = e + 1;
  // ---- nodal triads: lane 0..17 -> entry (node lane/9, index lane%9)
  if (lane < 18) {
    const int nd = lane < 9 ? a : b, idx = lane % 9, r = idx / 3, c = idx % 3;
    const double w = d.qw[nd], x = d.qx[nd], y = d.qy[nd], z = d.qz[nd];
    const double q[4] = {w, x, y, z};
    // R[r][c] of the unit quaternion: diagonal 1 - 2(q_j^2 + q_k^2), off-diagonal 2(q_r q_c -+ w q_k)
    double v;
    if (r == c) {
      const int j = (r + 1) % 3 + 1, k = (r + 2) % 3 + 1;
      v = 1.0 - 2.0 * (q[j] * q[j] + q[k] * q[k]);
    } else {
      const int k = 3 - r - c;                       // the third axis
      const double sgn = ((c - r + 3) % 3 == 1) ? -1.0 : 1.0;   // R[0][1] = 2(xy - wz), R[1][0] = 2(xy + wz)
      v = 2.0 * fma(q[r + 1], q[c + 1], sgn * w * q[k + 1]);
    }
    S.T[lane / 9][idx] = v;
  }
  __syncwarp();
  // ---- chord and rigid frame (scalar chain, lane-uniform)
  const double xa[3] = {d.px[a], d.py[a], d.pz[a]};
  const double dv[3] = {d.px[b] - xa[0], d.py[b] - xa[1], d.pz[b] - xa[2]};
  const double l2 = dot3(dv, dv);
  const double l = sqrt(l2);
  const double il = __drcp_rn(l);
  const double e1[3] = {dv[0] * il, dv[1] * il, dv[2] * il};
  const double qv[3] = {0.5 * (S.T[0][1] + S.T[1][1]), 0.5 * (S.T[0][4] + S.T[1][4]), 0.5 * (S.T[0][7] + S.T[1][7])};
  double v3[3];
  cross3(e1, qv, v3);
  const double iv = rsqrt(dot3(v3, v3));
  const double e3[3] = {v3[0] * iv, v3[1] * iv, v3[2] * iv};
  double e2[3];
  cross3(e3, e1, e2);
  if (lane < 9) {
    const int r = lane / 3, c = lane % 3;
    S.Rr[lane] = c == 0 ? e1[r] : (c == 1 ? e2[r] : e3[r]);
  }
  __syncwarp();
  // ---- R_r^T T for both nodes: lanes 0..17
  if (lane < 18) {
    const int nd = lane / 9, idx = lane % 9, i = idx / 3, j = idx % 3;
    const double* T = S.T[nd];
    S.Rab[nd][idx] = fma(S.Rr[i], T[j], fma(S.Rr[3 + i], T[3 + j], S.Rr[6 + i] * T[6 + j]));
  }
  __syncwarp();
  // ---- local rotations and Tsinv: lane 0 node a, lane 1 node b
  if (lane < 2) {
    double th[3], Ti[9];
    rotvec_of_mat(S.Rab[lane], th);
    tsinv_mat(th, Ti);
#pragma unroll
    for (int k = 0; k < 3; ++k) S.th[lane][k] = th[k];
#pragma unroll
    for (int k = 0; k < 9; ++k) S.Ti[lane][k] = Ti[k];
  }
  __syncwarp();
  const double u = (l2 - p.l0 * p.l0) / (l + p.l0);
  const double qb1 = dot3(e1, qv), qb2 = dot3(e2, qv);   // local components of q (third is 0)
  const double iq2 = __drcp_rn(qb2);
  const double* tha = S.th[0];
  const double* thb = S.th[1];
  const double* Tia = S.Ti[0];
  const double* Tib = S.Ti[1];
  const double* Ra = S.Rab[0];
  const double* Rb = S.Rab[1];
  const double* Rr = S.Rr;
  // local force vector f_l = K_l d_l
  const double ka = d.kel[4 * e], kt = d.kel[4 * e + 1], kb = d.kel[4 * e + 2];   // EA/l0, GJ/l0, EI/l0
  double fl[7];
  fl[0] = ka * u;
  fl[1] = kt * (tha[0] - thb[0]);
  fl[2] = kb * (4.0 * tha[1] + 2.0 * thb[1]);
  fl[3] = kb * (4.0 * tha[2] + 2.0 * thb[2]);
  fl[4] = -fl[1];
  fl[5] = kb * (2.0 * tha[1] + 4.0 * thb[1]);
  fl[6] = kb * (2.0 * tha[2] + 4.0 * thb[2]);
  auto& sB = S.B;
  auto& sH = S.H;

  // ---- column j of B (local components): lanes 0..11
  if (lane < 12) {
    const int j = lane;
    // G^T column j: spin of the rigid frame per unit local variation j
    double g0 = 0.0, g1 = 0.0, g2 = 0.0;
    if (j == 2) { g0 = qb1 * iq2 * il; g1 = il; }
    else if (j == 8) { g0 = -qb1 * iq2 * il; g1 = -il; }
    else if (j == 1) { g2 = -il; }
    else if (j == 7) { g2 = il; }
    else if (j == 3) { g0 = 0.5 * Ra[4] * iq2; }     // qa_bar = column 1 of Ra: (Ra[1], Ra[4], Ra[7])
    else if (j == 4) { g0 = -0.5 * Ra[1] * iq2; }
    else if (j == 9) { g0 = 0.5 * Rb[4] * iq2; }
    else if (j == 10) { g0 = -0.5 * Rb[1] * iq2; }
    double ca0 = -g0, ca1 = -g1, ca2 = -g2;   // (E_a - G^T) column j
    double cb0 = -g0, cb1 = -g1, cb2 = -g2;   // (E_b - G^T) column j
    if (j >= 3 && j < 6) { if (j == 3) ca0 += 1.0; else if (j == 4) ca1 += 1.0; else ca2 += 1.0; }
    if (j >= 9) { if (j == 9) cb0 += 1.0; else if (j == 10) cb1 += 1.0; else cb2 += 1.0; }
    sB[0][j] = (j == 0) ? -1.0 : ((j == 6) ? 1.0 : 0.0);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      sB[1 + r][j] = fma(Tia[3 * r], ca0, fma(Tia[3 * r + 1], ca1, Tia[3 * r + 2] * ca2));
      sB[4 + r][j] = fma(Tib[3 * r], cb0, fma(Tib[3 * r + 1], cb1, Tib[3 * r + 2] * cb2));
    }
  }
  __syncwarp();
  // ---- B E^T: global components, entries idx = lane + 32 t < 84
  double bg[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    int idx = lane + 32 * t;
    bg[t] = 0.0;
    if (idx < 84) {
      int k = idx / 12, col = idx % 12, s = col / 3, c = col % 3;
      bg[t] = fma(sB[k][3 * s], Rr[3 * c], fma(sB[k][3 * s + 1], Rr[3 * c + 1], sB[k][3 * s + 2] * Rr[3 * c + 2]));
    }
  }
  __syncwarp();
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    int idx = lane + 32 * t;
    if (idx < 84) sB[idx / 12][idx % 12] = bg[t];
  }
  __syncwarp();
  double* out = d.elem + (size_t)e * kElemStride;
  if constexpr (kMixed) {
    // ---- FP32 tangent: H = K_l (B E^T), K (upper triangle) = (B E^T)^T H
    const float ka32 = (float)ka, kt32 = (float)kt, kb32 = (float)kb;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      int idx = lane + 32 * t;
      if (idx < 84) S.B32[idx / 12][idx % 12] = (float)sB[idx / 12][idx % 12];
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      int idx = lane + 32 * t;
      if (idx < 84) {
        int k = idx / 12, col = idx % 12;
        const auto& b = S.B32;
        float h;
        switch (k) {
          case 0: h = ka32 * b[0][col]; break;
          case 1: h = kt32 * (b[1][col] - b[4][col]); break;
          case 4: h = kt32 * (b[4][col] - b[1][col]); break;
          case 2: h = kb32 * fmaf(4.0f, b[2][col], 2.0f * b[5][col]); break;
          case 5: h = kb32 * fmaf(2.0f, b[2][col], 4.0f * b[5][col]); break;
          case 3: h = kb32 * fmaf(4.0f, b[3][col], 2.0f * b[6][col]); break;
          default: h = kb32 * fmaf(2.0f, b[3][col], 4.0f * b[6][col]); break;
        }
        S.H32[k][col] = h;
      }
    }
    __syncwarp();
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      int idx = lane + 32 * t;
      if (idx < 78) {
        int i = c_up_i[idx], j = c_up_j[idx];
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < 7; ++k) s = fmaf(S.B32[k][i], S.H32[k][j], s);
        out[idx] = (double)s;
      }
    }
  } else {
    // ---- H = K_l (B E^T)
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      int idx = lane + 32 * t;
      if (idx < 84) {
        int k = idx / 12, col = idx % 12;
        double h;
        switch (k) {
          case 0: h = ka * sB[0][col]; break;
          case 1: h = kt * (sB[1][col] - sB[4][col]); break;
          case 4: h = kt * (sB[4][col] - sB[1][col]); break;
          case 2: h = kb * fma(4.0, sB[2][col], 2.0 * sB[5][col]); break;
          case 5: h = kb * fma(2.0, sB[2][col], 4.0 * sB[5][col]); break;
          case 3: h = kb * fma(4.0, sB[3][col], 2.0 * sB[6][col]); break;
          default: h = kb * fma(2.0, sB[3][col], 4.0 * sB[6][col]); break;
        }
        sH[k][col] = h;
      }
    }
    __syncwarp();
    // ---- K (upper triangle)
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      int idx = lane + 32 * t;
      if (idx < 78) {
        int i = c_up_i[idx], j = c_up_j[idx];
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < 7; ++k) s = fma(sB[k][i], sH[k][j], s);
        out[idx] = s;
      }
    }
  }
  // ---- F = (B E^T)^T f_l, FP64 in both modes
  if (lane < 12) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 7; ++k) s = fma(sB[k][lane], fl[k], s);
    out[78 + lane] = s;
  }
}

// The FP32 tangent unless the handle computes in FP64 or this solve fell back to FP64.
__device__ __forceinline__ bool mixed_tangent(const Params& p, const Dev& d) {
  return p.precision == kPrecisionMixed && !d.ctl->fp64_tangent;
}

__global__ void __launch_bounds__(32 * kWarpsPerElemBlock) element_kernel(Params p, Dev d) {
  __shared__ ElemShared sm[kWarpsPerElemBlock];
  pdl_enter();
  const int w = threadIdx.x >> 5;
  if (mixed_tangent(p, d)) element_warp<true>(p, d, blockIdx.x, w, sm[w]);
  else element_warp<false>(p, d, blockIdx.x, w, sm[w]);
}

// Batched element phase with kW warps per block (kW a multiple of kWarpsPerElemBlock): the plan's
// work units hold kWarpsPerElemBlock elements each, and a block takes kW / kWarpsPerElemBlock units
// at a time, one warp per element; each warp walks the plan's units independently (no block barrier).
// The element mapping (warps per block) is one of the batch's autotuned choices.
template <int kW>
__device__ __forceinline__ void element_batch_body(const Inst* __restrict__ tab, const Plan* __restrict__ plan) {
  static_assert(kW % kWarpsPerElemBlock == 0, "whole work units per block");
  constexpr int kUnits = kW / kWarpsPerElemBlock;
  __shared__ ElemShared sm[kW];
  __shared__ int s_pre[kMaxBatch + 1];
  pdl_enter();
  const int na = plan->n_act;
  const int total = plan->pre[PH_ELEM][na];
  if ((int)blockIdx.x * kUnits >= total) return;
  for (int i = threadIdx.x; i <= na; i += blockDim.x) s_pre[i] = plan->pre[PH_ELEM][i];
  __syncthreads();
  const int w = threadIdx.x >> 5;
  int j = 0;
  for (int u0 = blockIdx.x * kUnits; u0 < total; u0 += gridDim.x * kUnits) {
    const int u = u0 + w / kWarpsPerElemBlock;
    if (u >= total) break;
    while (s_pre[j + 1] <= u) ++j;                  // this warp's units come in increasing order
    const Inst& in = tab[plan->act[j]];
    if (mixed_tangent(in.p, in.d)) element_warp<true>(in.p, in.d, u - s_pre[j], w % kWarpsPerElemBlock, sm[w]);
    else element_warp<false>(in.p, in.d, u - s_pre[j], w % kWarpsPerElemBlock, sm[w]);
  }
}
__global__ void __launch_bounds__(64) element_batch_w2(const Inst* __restrict__ tab, const Plan* __restrict__ plan) {
  element_batch_body<2>(tab, plan);
}
__global__ void __launch_bounds__(128) element_batch_w4(const Inst* __restrict__ tab, const Plan* __restrict__ plan) {
  element_batch_body<4>(tab, plan);
}
__global__ void __launch_bounds__(256) element_batch_w8(const Inst* __restrict__ tab, const Plan* __restrict__ plan) {
  element_batch_body<8>(tab, plan);
}

void upload_element_tables() {
  unsigned char ui[78], uj[78];
  int n = 0;
  for (int i = 0; i < 12; ++i)
    for (int j = i; j < 12; ++j) { ui[n] = (unsigned char)i; uj[n] = (unsigned char)j; ++n; }
  cudaMemcpyToSymbol(c_up_i, ui, sizeof(ui));
  cudaMemcpyToSymbol(c_up_j, uj, sizeof(uj));
}

}  // namespace accfem
