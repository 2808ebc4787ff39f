// Assembly of the block-tridiagonal tangent over the free nodes (Eq. 20-23; Sec. III.C "assemble
// them into a tangent stiffness matrix") and its factorisation / multi-RHS solve by block cyclic
// reduction (6x6 blocks, depth ceil(log2 nf)).
//
// Free node f = node - k - 1 (f = 0 .. nf-1).  D_f = K_bb(elem node-1) + K_aa(elem node);
// U_f = K_{f,f+1} = K_ab(elem node); g_f = F(node) - F_a(node).  The prescribed DOFs are eliminated
// (Eq. 14-15), so the system is K dx = rhs on 6 nf unknowns.
//
// Cyclic reduction, level with stride s (s = 1, 2, 4, .. < nf): nodes j = s (mod 2s) are
// eliminated, nodes i = 0 (mod 2s) kept.  For eliminated j: P_j = D_j^{-1}, L_j = U_{j-s} P_j,
// R_j = U_j^T P_j.  For kept i: D_i -= R_{i-s} U_{i-s} + L_{i+s} U_i^T, U_i <- -L_{i+s} U_{i+s}.
// Solve: forward b_i -= R_{i-s} b_{i-s} + L_{i+s} b_{i+s} (kept), root x_0 = P_0 b_0, backward
// x_j = P_j b_j - L_j^T x_{j-s} - R_j^T x_{j+s} (eliminated).  Launches per factor-and-solve:
// the assembly kernel (with the level-1 eliminations), one bcr_level_kernel per level (kept-node update + next level's
// eliminations + forward RHS; root at the last level), one bcr_bwd_kernel per level.
#include "batch.cuh"

namespace accfem {

__device__ __forceinline__ int up_index(int i, int j) {   // upper triangle, row-major, i <= j < 12
  return i * 12 - (i * (i - 1)) / 2 + (j - i);
}
__device__ __forceinline__ double kval(const double* rec, int i, int j) {
  return i <= j ? rec[up_index(i, j)] : rec[up_index(j, i)];
}

// ------------------------------------------------------------------ constraint compaction
// Exclusive prefix over the 1024 threads of v; *total receives the sum (s_warp: 32 ints).
__device__ __forceinline__ int block_excl_scan_1024(int v, int* s_warp, int* total) {
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += t;
  }
  __syncthreads();
  if (lane == 31) s_warp[w] = x;
  __syncthreads();
  if (w == 0) {
    int y = s_warp[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += t;
    }
    s_warp[lane] = y;
  }
  __syncthreads();
  *total = s_warp[31];
  return x - v + (w > 0 ? s_warp[w - 1] : 0);
}

// One CTA: exclusive scan of the per-node row counts, row arrays in (node, triangle) order,
// comparison with the previous iteration's rows (flags carried by identity), the working set of
// the contact solve, copy to "previous".  Working set: rows active in the previous iteration, rows
// violated by an applied step in this solve (they stay), and rows whose gap is at most ws_gap (all
// rows in frame mode, where every iteration is a reported state and solves the QP of Eq. 23 whole);
// when that exceeds the working-set cap, the near rows with the smallest gaps up to the cap; slots
// follow the row order.
__device__ __forceinline__ void compact_body(const Params& p, const Dev& d) {
  __shared__ int s_warp[32];
  __shared__ int s_same;
  Ctl* ctl = d.ctl;
  if (ctl->status != 0 || ctl->converged) return;
  const int nf = ctl->nf;
  const int tid = threadIdx.x;
  const int per = (nf + 1023) / 1024;
  const int f0 = tid * per, f1 = min(f0 + per, nf);
  if (p.contact_model == kContactSegment) {
    // a contact at a shared node appears on both elements (s = 1 of element f - 1, s = 0 of element
    // f, the same wall point): keep the lower element's row
    for (int f = f0; f < f1; ++f) {
      unsigned keep = 0u;
      const int nc = d.ncon[f];
      for (int r = 0; r < nc; ++r) {
        const int src = f * kListCap + r;
        bool drop = false;
        if (f > 0 && d.con_s[src] == 0.0) {
          const int np = d.ncon[f - 1];
          for (int q = 0; q < np && !drop; ++q) {
            const int o = (f - 1) * kListCap + q;
            if (d.con_s[o] != 1.0) continue;
            const double dx = d.con_pt[3 * o] - d.con_pt[3 * src], dy = d.con_pt[3 * o + 1] - d.con_pt[3 * src + 1],
                         dz = d.con_pt[3 * o + 2] - d.con_pt[3 * src + 2];
            drop = sqrt(dx * dx + dy * dy + dz * dz) <= 1e-12;
          }
        }
        if (!drop) keep |= 1u << r;
      }
      d.con_keep[f] = (int)keep;
    }
    __syncthreads();
    for (int f = f0; f < f1; ++f) {              // compact each element's list in place
      const unsigned keep = (unsigned)d.con_keep[f];
      int o = 0;
      for (int r = 0; r < d.ncon[f]; ++r) {
        if (!(keep & (1u << r))) continue;
        const int a = f * kListCap + r, b = f * kListCap + o;
        if (a != b) {
          d.con_tri[b] = d.con_tri[a];
          d.con_gap[b] = d.con_gap[a];
          d.con_s[b] = d.con_s[a];
          for (int c = 0; c < 3; ++c) { d.con_pt[3 * b + c] = d.con_pt[3 * a + c]; d.con_n[3 * b + c] = d.con_n[3 * a + c]; }
        }
        ++o;
      }
      d.ncon[f] = o;
    }
  }
  int loc = 0;
  for (int f = f0; f < f1; ++f) loc += d.ncon[f];
  if (tid == 0) s_same = 1;
  int m = 0;
  const int excl = block_excl_scan_1024(loc, s_warp, &m);
  if (m > p.m_cap) {
    if (tid == 0) flag_capacity(ctl, CAP_ROWS);
    return;
  }
  int row = excl;
  for (int f = f0; f < f1; ++f) {             // row ranges and the node of every row
    d.c_first[f] = row;
    const int nc = d.ncon[f];
    for (int r = 0; r < nc; ++r, ++row) d.c_node[row] = f;
  }
  if (tid == 0) d.c_first[nf] = m;
  __syncthreads();
  for (int r = tid; r < m; r += 1024) {       // row payloads, one thread per row
    const int f = d.c_node[r];
    const int src = f * kListCap + (r - d.c_first[f]);
    d.c_tri[r] = d.con_tri[src];
    double n[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      d.c_pt[3 * r + c] = d.con_pt[src * 3 + c];
      n[c] = d.con_n[src * 3 + c];
      d.c_n[3 * r + c] = n[c];
    }
    d.c_gap[r] = d.con_gap[src];
    if (p.contact_model == kContactSegment) {
      // Eq. 4-6 in the element frame: du(xi) = R_r N(xi) [R_r^T du_a; R_r^T du_b], axial weights P1, P2
      // along the chord e1 and transverse weights P3, P4 across it, so
      // n^T du(xi) = (P3 n + (P1 - P3)(n.e1) e1) . du_a + (P4 n + (P2 - P4)(n.e1) e1) . du_b
      const int na = ctl->k + f, nb = na + 1;
      double e1[3] = {d.px[nb] - d.px[na], d.py[nb] - d.py[na], d.pz[nb] - d.pz[na]};
      const double il = 1.0 / sqrt(dot3(e1, e1));
      e1[0] *= il; e1[1] *= il; e1[2] *= il;
      const double rr = d.con_s[src];
      const double P1 = 1.0 - rr, P2 = rr, P3 = 1.0 - 3.0 * rr * rr + 2.0 * rr * rr * rr, P4 = 3.0 * rr * rr - 2.0 * rr * rr * rr;
      const double ne = dot3(n, e1);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        d.c_w1[3 * r + c] = P4 * n[c] + (P2 - P4) * ne * e1[c];    // the element's far node (free node f)
        d.c_w2[3 * r + c] = P3 * n[c] + (P1 - P3) * ne * e1[c];    // its near node (free node f - 1)
      }
      d.c_node2[r] = f > 0 ? f - 1 : -1;
      d.c_s[r] = rr;
    } else {
#pragma unroll
      for (int c = 0; c < 3; ++c) { d.c_w1[3 * r + c] = n[c]; d.c_w2[3 * r + c] = 0.0; }
      d.c_node2[r] = -1;
      d.c_s[r] = 0.0;
    }
  }
  __syncthreads();
  const int mp = ctl->m_prev;
  // flags of the same row (node, triangle) in the previous iteration; -1 for a new row.  The node's
  // previous rows are [p_first[f], p_first[f+1]) (at most kListCap; none before the first compaction)
  for (int r = tid; r < m; r += 1024) {
    const int nd = d.c_node[r], tr = d.c_tri[r];
    int found = -1;
    if (mp >= 0) {
      const int q0 = d.p_first[nd], q1 = d.p_first[nd + 1];
#pragma unroll 4
      for (int q = q0; q < q1; ++q)
        if (d.p_tri[q] == tr) found = q;
    }
    d.init_flag[r] = found >= 0 ? d.p_flag[found] : -1;
  }
  if (mp != m) {
    if (tid == 0) s_same = 0;
  } else {
    for (int r = tid; r < m; r += 1024)
      if (d.p_node[r] != d.c_node[r] || d.p_tri[r] != d.c_tri[r]) s_same = 0;
  }
  __syncthreads();
  // working set: contiguous row chunks per thread, slots in row order
  const int rper = (m + 1023) / 1024;
  const int r0 = min(tid * rper, m), r1 = min(r0 + rper, m);
  const int keep_mask = RF_ACTIVE | RF_VIOLATED | RF_STICKY;
  // no applied step of this iteration moves a node farther than the limiter's bound, at most
  // min(1.5 rho, beta0): rows with a larger gap cannot be violated by it
  double ws_gap = fmin(p.ws_gap, fmin(1.5 * ctl->rho, p.beta0));
  int nw = 0;
  for (int r = r0; r < r1; ++r) {
    const int fl = d.init_flag[r];
    nw += (p.ws_all || (fl > 0 && (fl & keep_mask)) || d.c_gap[r] <= ws_gap) ? 1 : 0;
  }
  int mc = 0;
  int slot = block_excl_scan_1024(nw, s_warp, &mc);
  if (mc > p.ws_cap && !p.ws_all) {
    // more near rows than the cap: keep the active and violated rows and, of the near rows, those with
    // the smallest gaps (the threshold bisected down until the count fits); rows left out are still
    // checked against the applied step and join when violated
    int mand = 0, cnt = 0;
    for (int r = r0; r < r1; ++r) {
      const int fl = d.init_flag[r];
      mand += (fl > 0 && (fl & keep_mask)) ? 1 : 0;
    }
    block_excl_scan_1024(mand, s_warp, &cnt);
    if (cnt > p.ws_cap) {
      if (tid == 0) flag_capacity(ctl, CAP_WORKING);
      return;
    }
    double lo = -1.0, hi = ws_gap;          // count(lo) <= cap < count(hi)
    for (int it = 0; it < 48; ++it) {
      const double mid = 0.5 * (lo + hi);
      int k = 0;
      for (int r = r0; r < r1; ++r) {
        const int fl = d.init_flag[r];
        k += ((fl > 0 && (fl & keep_mask)) || d.c_gap[r] <= mid) ? 1 : 0;
      }
      int tot = 0;
      block_excl_scan_1024(k, s_warp, &tot);
      if (tot <= p.ws_cap) lo = mid; else hi = mid;
    }
    ws_gap = lo;
    nw = 0;
    for (int r = r0; r < r1; ++r) {
      const int fl = d.init_flag[r];
      nw += ((fl > 0 && (fl & keep_mask)) || d.c_gap[r] <= ws_gap) ? 1 : 0;
    }
    slot = block_excl_scan_1024(nw, s_warp, &mc);
  }
  if (mc > p.ws_cap) {
    if (tid == 0) flag_capacity(ctl, CAP_WORKING);
    return;
  }
  for (int r = r0; r < r1; ++r) {
    const int fl = d.init_flag[r];
    if (p.ws_all || (fl > 0 && (fl & keep_mask)) || d.c_gap[r] <= ws_gap) {
      d.wrow[slot] = r;
      d.rslot[r] = slot++;
    } else {
      d.rslot[r] = -1;
    }
  }
  __syncthreads();
  for (int f = tid; f <= nf; f += 1024) d.p_first[f] = d.c_first[f];
  for (int r = tid; r < m; r += 1024) {
    const int fl = d.init_flag[r];
    d.p_node[r] = d.c_node[r];
    d.p_tri[r] = d.c_tri[r];
    d.p_flag[r] = d.rslot[r] >= 0 ? (RF_WORKING | ((fl > 0 && (fl & (RF_VIOLATED | RF_STICKY))) ? RF_STICKY : 0)) : 0;
  }
  if (tid == 0) { ctl->same_set = s_same; ctl->m = m; ctl->m_prev = m; ctl->mc = mc; }
}

__global__ void __launch_bounds__(1024) compact_kernel(Params p, Dev d) {
  pdl_enter();
  compact_body(p, d);
}

__global__ void __launch_bounds__(1024) compact_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan) {
  for_units(tab, plan, PH_COMPACT, [](const Inst& in, int, int) { compact_body(in.p, in.d); });
}

// ------------------------------------------------------------------ assembly
__device__ bool team_inverse6(double* sA, int tid);
__device__ __forceinline__ void team_lr6(const double* sX, const double* sY, const double* sP, double* P, double* L,
                                         double* R, int tid);

// Assembly and RHS columns of one free node (blocks (node, y), 32 x 6 threads): D, U and g = F - F_a
// with the tip load of Eq. 16-18, then RHS columns 0 = -g and 1 + k = A^T e_row for the row of
// working-set slot k (block y takes the column chunks y, y + kRhsSplit, ...).  Block y = 0 of an
// odd node f also does its elimination at the first level of the reduction: both couplings come
// from its own element records (U_{f-1} = K_{f-1,f} of the element before the node, U_f of the one
// after it), so P_f = D_f^{-1}, L_f = U_{f-1} P_f and R_f = U_f^T P_f need no other block.
__device__ __forceinline__ void assemble_rhs_body(const Params& p, const Dev& d, int bx, int by) {
  __shared__ double s_g[6];
  __shared__ double sA[36], sXl[36], sYr[36];
  Ctl* ctl = d.ctl;
  if (ctl->status != 0 || ctl->converged) return;
  const int f = bx;
  const int nf = ctl->nf;
  if (f >= nf) return;
  const int node = ctl->k + 1 + f;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  const double* eb = d.elem + (size_t)(node - 1) * kElemStride;
  const double* ea = d.elem + (size_t)node * kElemStride;
  const bool has_a = node < p.M;
  const bool elim1 = by == 0 && (f & 1);
  if (tid < 36 && by == 0) {
    int r = tid / 6, c = tid % 6;
    double v = kval(eb, 6 + r, 6 + c);
    if (has_a) v += kval(ea, r, c);
    d.D[(size_t)f * 36 + tid] = v;
    sA[tid] = v;
  } else if (tid >= 36 && tid < 72 && by == 0) {
    int q = tid - 36, r = q / 6, c = q % 6;
    const double u = has_a ? kval(ea, r, 6 + c) : 0.0;
    d.U[(size_t)f * 36 + q] = u;
    sYr[q] = u;                                     // U_f = K_{f, f+1} (0 at the tip)
  } else if (elim1 && tid >= 78 && tid < 114) {
    int q = tid - 78, r = q / 6, c = q % 6;
    sXl[q] = kval(eb, r, 6 + c);                    // U_{f-1} = K_{f-1, f}
  } else if (tid >= 72 && tid < 78) {
    int c = tid - 72;
    double F = eb[78 + 6 + c] + (has_a ? ea[78 + c] : 0.0);
    double Fa = 0.0;
    if (node == p.M) {
      double T[9];
      quat_to_mat(d.qw[node], d.qx[node], d.qy[node], d.qz[node], T);
      double fl[3] = {0.0, 0.0, 0.0}, ml[3] = {0.0, 0.0, 0.0};
      if (ctl->load_mode == 0) {
        double st = 0.0, ss = 0.0, sc = 0.0;
        for (int j = 0; j < p.n_cables; ++j) {
          st += ctl->tension[j];
          ss += ctl->tension[j] * p.cable_sin[j];
          sc += ctl->tension[j] * p.cable_cos[j];
        }
        fl[0] = -st; ml[1] = -p.r_c * ss; ml[2] = p.r_c * sc;
      } else {
        for (int a2 = 0; a2 < 3; ++a2) { fl[a2] = ctl->tip_f[a2]; ml[a2] = ctl->tip_m[a2]; }
      }
      if (ctl->load_mode == 1) {
        Fa = c < 3 ? fl[c] : ml[c - 3];
      } else {
        const double* v = c < 3 ? fl : ml;
        int r = c % 3;
        Fa = fma(T[3 * r], v[0], fma(T[3 * r + 1], v[1], T[3 * r + 2] * v[2]));
      }
    }
    s_g[c] = F - Fa;
    if (by == 0) d.g[(size_t)f * 6 + c] = F - Fa;
  }
  if (elim1) {                                      // first-level elimination of node f
    const bool ok = team_inverse6(sA, tid);  // begins with a barrier
    if (!ok) {
      if (tid == 0) atomicCAS(&ctl->status, 0, ST_NOT_SPD);
    } else {                                        // P_f, L_f = U_{f-1} P_f, R_f = U_f^T P_f
      team_lr6(sXl, sYr, sA, d.P + (size_t)f * 36, d.Lm + (size_t)f * 36, d.Rm + (size_t)f * 36, tid);
    }
  }
  __syncthreads();
  const int c = threadIdx.y;
  const int nrhs = ctl->mc + 1;
  for (int r = by * 32 + threadIdx.x; r < nrhs; r += 32 * kRhsSplit) {
    double v;
    if (r == 0) {
      v = -s_g[c];
    } else {
      const int row = d.wrow[r - 1];
      if (c >= 3) v = 0.0;
      else if (p.contact_model == kContactNode) v = d.c_node[row] == f ? d.c_w1[3 * row + c] : 0.0;
      else v = d.c_node[row] == f ? d.c_w1[3 * row + c] : (d.c_node2[row] == f ? d.c_w2[3 * row + c] : 0.0);
    }
    d.B[((size_t)f * 6 + c) * p.nrhs_cap + r] = v;
  }
}

__global__ void __launch_bounds__(192) assemble_rhs_kernel(Params p, Dev d) {
  pdl_enter();
  assemble_rhs_body(p, d, blockIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(192) assemble_rhs_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan) {
  for_units(tab, plan, PH_ASM, [](const Inst& in, int bx, int by) { assemble_rhs_body(in.p, in.d, bx, by); });
}

// ------------------------------------------------------------------ 6x6 helpers
// The FP64 pipe of an SMSP takes a warp instruction every 64 cycles whatever its lane mask, so the
// helpers below give each class of entries (each with its own formula) a warp of its own: no warp
// runs the instructions of another class, and the classes run on different SMSPs in parallel (warp
// w of a block sits on SMSP w mod 4).  The arithmetic of every entry is the same as one thread per
// entry would do.

// Named barrier `id` over n threads: the producers arrive without waiting, the consumers wait (the
// producers' earlier shared-memory writes are then visible to the consumers).
__device__ __forceinline__ void named_arrive(int id, int n) { asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory"); }
__device__ __forceinline__ void named_sync(int id, int n) { asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory"); }

// In-place Gauss-Jordan inverse of the SPD matrix in sA (6x6, row-major), called by every thread of
// a block of at least 128 threads (named barrier 1 is used between warps 0 and 1).  Returns false
// (for all threads) when a pivot is not positive.  2x2 block pivots (DOFs k, k + 1 for k = 0, 2,
// 4): the block's inverse Binv from its determinant, one reciprocal for two DOFs; the block is SPD
// exactly when its two scalar pivots (a, det / a) are positive.  Entries of a pivot step: the 8 of
// the pivot rows outside the pivot columns (warp 1: Binv times the two rows, which it also hands to
// warp 0), the 16 outside the pivot rows and columns (warp 0: the entry less the row's two pivot-
// column entries times those scaled rows), the 8 of the pivot columns outside the pivot rows (warp
// 2) and the 4 of the block (warp 3).  Each lane forms only the entries of Binv its formula uses.
__device__ bool team_inverse6(double* sA, int tid) {
  __shared__ double s_piv[2][4];                   // the scaled pivot rows, outside the pivot columns
  const int w = tid >> 5, l = tid & 31;
  for (int k = 0; k < 6; k += 2) {
    __syncthreads();
    const double a = sA[k * 6 + k], b = sA[k * 6 + k + 1], b2 = sA[(k + 1) * 6 + k], cc = sA[(k + 1) * 6 + k + 1];
    const double det = fma(a, cc, -(b * b2));
    if (!(a > 0.0) || !(det > 0.0)) return false;
    // this thread's entry (r, c) of the step, r = -1 for none; t -> t + 2 (t >= k) maps 0..3 onto
    // the indices outside the pivot pair
    int r = -1, c = -1;
    if (w == 0 && l < 16) {
      r = l >> 2; c = l & 3;
      r += r >= k ? 2 : 0; c += c >= k ? 2 : 0;
    } else if (w == 1 && l < 8) {
      r = k + (l >> 2); c = l & 3;
      c += c >= k ? 2 : 0;
    } else if (w == 2 && l < 8) {
      r = l >> 1; c = k + (l & 1);
      r += r >= k ? 2 : 0;
    } else if (w == 3 && l < 4) {
      r = k + (l >> 1); c = k + (l & 1);
    }
    double v = 0.0;
    if (w == 1) {                                    // pivot rows: Binv [a_kc; a_k+1,c]
      if (r >= 0) {
        const double rd = __drcp_rn(det);
        const double e0 = (r == k ? cc : -b2) * rd, e1 = (r == k ? -b : a) * rd;
        v = fma(e0, sA[k * 6 + c], e1 * sA[(k + 1) * 6 + c]);
        s_piv[l >> 2][l & 3] = v;
      }
      named_arrive(1, 64);
    } else if (w == 0) {                             // a_rc - [a_rk, a_r,k+1] Binv [a_kc; a_k+1,c]
      named_sync(1, 64);
      if (r >= 0) v = fma(-sA[r * 6 + k], s_piv[0][l & 3], fma(-sA[r * 6 + k + 1], s_piv[1][l & 3], sA[r * 6 + c]));
    } else if (r >= 0) {
      const double rd = __drcp_rn(det);
      if (w == 2) {                                  // pivot columns: -[a_rk, a_r,k+1] Binv[:, c]
        const double e0 = (c == k ? cc : -b) * rd, e1 = (c == k ? -b2 : a) * rd;
        v = -fma(sA[r * 6 + k], e0, sA[r * 6 + k + 1] * e1);
      } else {                                       // the block: Binv
        v = (r == k ? (c == k ? cc : -b) : (c == k ? -b2 : a)) * rd;
      }
    }
    __syncthreads();
    if (r >= 0) sA[r * 6 + c] = v;
  }
  __syncthreads();
  return true;
}

// The products of an elimination with P = sP (6x6 row-major, shared): L = X P and R = Y^T P (X, Y
// in shared memory) to L and R, P itself to P (global).  Entries 0..31 of L in warp 0, of R in warp
// 1, the last four of each in warp 2, so that every SMSP runs at most six FMA instructions.
__device__ __forceinline__ void team_lr6(const double* sX, const double* sY, const double* sP, double* P, double* L,
                                         double* R, int tid) {
  const int w = tid >> 5, l = tid & 31;
  int t = -1;                                        // 0..35: entry of L, 36..71: entry t - 36 of R
  if (w == 0) t = l;
  else if (w == 1) t = 36 + l;
  else if (w == 2 && l < 8) t = l < 4 ? 32 + l : 64 + l;
  if (t < 0) return;
  const bool isL = t < 36;
  const int q = isL ? t : t - 36, r = q / 6, c = q % 6;
  const double* A = isL ? sX + r * 6 : sY + r;       // row r of X, or column r of Y
  const int st = isL ? 1 : 6;
  double v = 0.0;
#pragma unroll
  for (int k = 0; k < 6; ++k) v = fma(A[k * st], sP[k * 6 + c], v);
  if (isL) {
    P[q] = sP[q];
    L[q] = v;
  } else {
    R[q] = v;
  }
}

// Level s of the reduction, fused with the elimination at level 2s.  Blocks (kept node i = 2 s x,
// y), 192 threads.  Block y == 0: Schur update of D_i and U_i (kept nodes i: D_i and U_i as above);
// when i = 2s (mod 4s) it then eliminates i at level 2s: its new left coupling
// U_{i-2s} <- -L_{i-s} U_{i-s} is rebuilt from level-s data, P_i = D_i^{-1}, L_i = U_{i-2s} P_i,
// R_i = U_i^T P_i.  Blocks y >= 1 apply the level-s forward reduction to their RHS chunks (chunk
// y - 1 + kRhsSplit q).  When 2s >= nf only node 0 is kept: every block inverts D_0 itself (root)
// and blocks y >= 1 solve x_0 = P_0 b_0 for their chunks.
// kLate: nf comes from the launch, and the control block's status is read beside the 6x6 block
// loads (tested after the first barrier, before any store), so that those loads need not wait for
// it (the RHS loads still wait for the column count).  Otherwise the caller has tested the status
// and read nf.
template <bool kLate>
__device__ __forceinline__ void bcr_level_run(const Params& p, const Dev& d, int nf, int bx, int by, int s) {
  __shared__ double sRl[36], sUl[36], sLl[36], sLr[36], sUi[36], sUr[36], sA[36], sX[36], sY[36];
  __shared__ int s_go;
  Ctl* ctl = d.ctl;
  const int i = 2 * s * bx;
  if (i >= nf) return;
  const int tid = threadIdx.x;
  const bool hl = i >= s, hr = i + s < nf, hr2 = i + 2 * s < nf;
  const bool root = 2 * s >= nf;                       // only node 0 remains after this level
  const bool elim2 = !root && (i % (4 * s)) == 2 * s;   // i is eliminated at level 2s
  // RHS values of this block's first column chunk, loaded with the blocks so that the two
  // latencies overlap (the columns of nodes i +- s are not written at this level)
  const int lane = tid & 31, c = tid >> 5;
  if (kLate && tid == 0) s_go = ctl->status == 0 && !ctl->converged;
  const int nrhs = ctl->mc + 1;
  const size_t ld = p.nrhs_cap;
  // block y == 0 does the 6x6 block work only; blocks y >= 1 reduce the RHS column chunks y - 1,
  // y - 1 + kRhsSplit, .. (so the launch takes the longer of the two paths, not their sum)
  const int chunk0 = by > 0 ? (by - 1) * 32 : (1 << 30);
  const int r_first = chunk0 + lane;
  double b_own = 0.0, b_l[6], b_r[6];
  auto load_rhs = [&](int r) {
    b_own = d.B[((size_t)i * 6 + c) * ld + r];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      b_l[k] = hl ? d.B[((size_t)(i - s) * 6 + k) * ld + r] : 0.0;
      b_r[k] = hr ? d.B[((size_t)(i + s) * 6 + k) * ld + r] : 0.0;
    }
  };
  if (r_first < nrhs) load_rhs(r_first);
  const double d_own = (tid < 36 && (by == 0 || root)) ? d.D[(size_t)i * 36 + tid] : 0.0;   // with the blocks
  if (tid < 36) {
    sRl[tid] = hl ? d.Rm[(size_t)(i - s) * 36 + tid] : 0.0;
    sUl[tid] = hl ? d.U[(size_t)(i - s) * 36 + tid] : 0.0;
    sLl[tid] = (hl && elim2) ? d.Lm[(size_t)(i - s) * 36 + tid] : 0.0;
    sLr[tid] = hr ? d.Lm[(size_t)(i + s) * 36 + tid] : 0.0;
    sUi[tid] = hr ? d.U[(size_t)i * 36 + tid] : 0.0;
    sUr[tid] = hr2 ? d.U[(size_t)(i + s) * 36 + tid] : 0.0;
  }
  __syncthreads();
  if (kLate && !s_go) return;
  const bool matrix = by == 0 || root;
  // the root's D_0 and U_0 are read by every block of this level and needed by no later step: only
  // non-root levels store the updated blocks (for the next level's kernel)
  const bool store = by == 0 && !root;
  if (tid < 36 && matrix) {                          // Schur update of D_i (warp 0, lanes 0..3 of warp 1)
    const int r = tid / 6, c = tid % 6;
    double dd = d_own;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      dd = fma(-sRl[r * 6 + k], sUl[k * 6 + c], dd);
      dd = fma(-sLr[r * 6 + k], sUi[c * 6 + k], dd);
    }
    sA[tid] = dd;
    if (store) d.D[(size_t)i * 36 + tid] = dd;
  } else if (matrix && (tid >> 5) >= 2 && (tid >> 5) <= 3) {
    // beside it, in warps 2 and 3: the new U_i = K_{i, i+2s} = -L_{i+s} U_{i+s} (products 0..35)
    // and, for an elimination at level 2s, the new left coupling K_{i-2s, i} = -L_{i-s} U_{i-s}
    // (products 36..71; node i-s was eliminated at level s): warp 2 takes products lane and 64 +
    // lane, warp 3 products 32 + lane
    const int nprod = (elim2 && by == 0) ? 72 : 36;
    for (int t = (tid >> 5) == 2 ? lane : 32 + lane; t < nprod; t += 64) {
      const bool isU = t < 36;
      const int q = isU ? t : t - 36, r = q / 6, c = q % 6;
      const double* A = isU ? sLr : sLl;
      const double* B = isU ? sUr : sUl;
      double v = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) v = fma(-A[r * 6 + k], B[k * 6 + c], v);
      if (isU) {
        sY[q] = hr2 ? v : 0.0;
        if (store && hr) d.U[(size_t)i * 36 + q] = hr2 ? v : 0.0;
      } else {
        sX[q] = v;
      }
    }
  }
  if (elim2 && by == 0) {
    const bool ok = team_inverse6(sA, tid);   // begins with a barrier
    if (!ok) {
      if (tid == 0) atomicCAS(&ctl->status, 0, ST_NOT_SPD);
    } else {                                         // P_i, L_i = U_{i-2s} P_i, R_i = U_i^T P_i
      team_lr6(sX, sY, sA, d.P + (size_t)i * 36, d.Lm + (size_t)i * 36, d.Rm + (size_t)i * 36, tid);
    }
  }
  // forward reduction of level s: b_i -= R_{i-s} b_{i-s} + L_{i+s} b_{i+s}
  if (!root) {
    for (int r = r_first; r < nrhs; r += 32 * kRhsSplit) {
      if (r != r_first) load_rhs(r);
      double acc = b_own;
      if (hl) {
#pragma unroll
        for (int k = 0; k < 6; ++k) acc = fma(-sRl[c * 6 + k], b_l[k], acc);
      }
      if (hr) {
#pragma unroll
        for (int k = 0; k < 6; ++k) acc = fma(-sLr[c * 6 + k], b_r[k], acc);
      }
      d.B[((size_t)i * 6 + c) * ld + r] = acc;
    }
    return;
  }
  // root: node 0 after its last update; every block inverts D_0 and solves its chunks
  __syncthreads();
  const bool ok = team_inverse6(sA, tid);
  if (!ok) {
    if (tid == 0) atomicCAS(&ctl->status, 0, ST_NOT_SPD);
    return;
  }
  if (tid < 36 && by == 0) d.P[tid] = sA[tid];
  for (int r0 = chunk0; r0 < nrhs; r0 += 32 * kRhsSplit) {
    const int r = r0 + lane;
    const bool act = r < nrhs;
    double acc0 = 0.0;
    if (act) {
      if (r0 != chunk0) load_rhs(r);                // i = 0 here; the first chunk was loaded above
      acc0 = b_own;
      if (hr) {
#pragma unroll
        for (int k = 0; k < 6; ++k) acc0 = fma(-sLr[c * 6 + k], b_r[k], acc0);
      }
    }
    __syncthreads();
    if (act) d.B[(size_t)c * ld + r] = acc0;          // b_0 after the last forward step
    __syncthreads();
    double bb[6];
    if (act)
#pragma unroll
      for (int k = 0; k < 6; ++k) bb[k] = d.B[(size_t)k * ld + r];
    __syncthreads();
    if (act) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) acc = fma(sA[c * 6 + k], bb[k], acc);
      d.B[(size_t)c * ld + r] = acc;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void bcr_level_body(const Params& p, const Dev& d, int bx, int by, int s) {
  const Ctl* ctl = d.ctl;
  if (ctl->status != 0 || ctl->converged) return;
  bcr_level_run<false>(p, d, ctl->nf, bx, by, s);
}

// nf: the free nodes of the Newton graph this launch belongs to (fixed during a solve)
__global__ void __launch_bounds__(192) bcr_level_kernel(Params p, Dev d, int s, int nf) {
  pdl_enter();
  bcr_level_run<true>(p, d, nf, blockIdx.x, blockIdx.y, s);
}

// level j (stride 2^j) of every iterating instance
__global__ void __launch_bounds__(192, 3) bcr_level_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan, int j) {
  for_units(tab, plan, PH_LEV0 + j, [j](const Inst& in, int bx, int by) { bcr_level_body(in.p, in.d, bx, by, 1 << j); });
}

// Back substitution at stride s for eliminated nodes j = s + 2 s blockIdx.x.  96 threads: 16 columns
// x 6 components, one warp per SMSP (a warp's FP64 instruction holds its SMSP's FP64 pipe for 64
// cycles, so two warps on one SMSP would serialise); block y takes the 16-column chunks y,
// y + kBwdSplit, ...
// kLate as in bcr_level_run.
template <bool kLate>
__device__ __forceinline__ void bcr_bwd_run(const Params& p, const Dev& d, int nf, int bx, int by, int s) {
  __shared__ double sP[36], sL[36], sR[36];
  __shared__ int s_go;
  const Ctl* ctl = d.ctl;
  const int j = s + 2 * s * bx;
  if (j >= nf) return;
  const int tid = threadIdx.x;
  const bool hr = j + s < nf;
  const int lane = tid & 15, c = tid >> 4;
  if (kLate && tid == 0) s_go = ctl->status == 0 && !ctl->converged;
  const int nrhs = ctl->mc + 1;
  const size_t ld = p.nrhs_cap;
  // b_j, x_{j-s}, x_{j+s} of the column this thread reads in a chunk (the first chunk's loaded with
  // the blocks, so that the two latencies overlap; x_{j+-s} are not written at this level)
  double b[6], xl[6], xr[6];
  auto load = [&](int r) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      b[k] = d.B[((size_t)j * 6 + k) * ld + r];
      xl[k] = d.B[((size_t)(j - s) * 6 + k) * ld + r];
      xr[k] = hr ? d.B[((size_t)(j + s) * 6 + k) * ld + r] : 0.0;
    }
  };
  if (by * 16 + lane < nrhs) load(by * 16 + lane);
  if (tid < 36) {
    sP[tid] = d.P[(size_t)j * 36 + tid];
    sL[tid] = d.Lm[(size_t)j * 36 + tid];
    sR[tid] = hr ? d.Rm[(size_t)j * 36 + tid] : 0.0;
  }
  __syncthreads();
  if (kLate && !s_go) return;
  for (int r0 = by * 16; r0 < nrhs; r0 += 16 * kBwdSplit) {
    const int r = r0 + lane;
    const bool act = r < nrhs;
    if (r0 != by * 16) {
      if (act) load(r);
      __syncthreads();                          // every read of b_j's column before its writes
    }
    if (act) {
      double acc = 0.0;
#pragma unroll
      for (int k = 0; k < 6; ++k) acc = fma(sP[c * 6 + k], b[k], acc);
#pragma unroll
      for (int k = 0; k < 6; ++k) acc = fma(-sL[k * 6 + c], xl[k], acc);    // - L_j^T x_{j-s}
      if (hr) {
#pragma unroll
        for (int k = 0; k < 6; ++k) acc = fma(-sR[k * 6 + c], xr[k], acc);  // - R_j^T x_{j+s}
      }
      d.B[((size_t)j * 6 + c) * ld + r] = acc;
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void bcr_bwd_body(const Params& p, const Dev& d, int bx, int by, int s) {
  const Ctl* ctl = d.ctl;
  if (ctl->status != 0 || ctl->converged) return;
  bcr_bwd_run<false>(p, d, ctl->nf, bx, by, s);
}

__global__ void __launch_bounds__(96) bcr_bwd_kernel(Params p, Dev d, int s, int nf) {
  pdl_enter();
  bcr_bwd_run<true>(p, d, nf, blockIdx.x, blockIdx.y, s);
}

__global__ void __launch_bounds__(96) bcr_bwd_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan, int j) {
  for_units(tab, plan, PH_BWD0 + j, [j](const Inst& in, int bx, int by) { bcr_bwd_body(in.p, in.d, bx, by, 1 << j); });
}

}  // namespace accfem
