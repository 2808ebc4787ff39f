// Robot-node vs lumen-triangle collision detection (Eq. 3-10; Sec. III.C: nodes are matched
// with the triangles in parallel and each match yields its constraint).  One warp per free node.
//
// Constraint rule (identical to an all-pairs FP64 scan): with c_t the closest point of triangle
// t to the node p, d_t = |c_t - p| and g the triangle of smallest d_t (lowest index on ties),
// (node, t) is a constraint row when d_t <= r_o + activation_gap and the node lies over t's face
// (plane projection inside the triangle enlarged by the barycentric margin kFaceBand), or t == g.
// The row's normal is the face normal when the projection is inside the triangle itself, else
// along c_t - p (edge/vertex point).  Rows with the same closest point (within 1e-12 m) are
// merged, keeping the lowest index.
//
// Work split: triangles are binned by centroid in a uniform grid; a node scans the cells of the
// box p +- (r_o + gap + max triangle radius) that come within that distance of p (the box's corner
// cells often do not: about a quarter of the slots).  A triangle whose FP32 bounding sphere stays beyond
// the activation distance (+ eps_d) is skipped.  Pass 1 computes FP32 distances (coordinates
// relative to the cell centre, so |x| is a few mm and the FP32 error a few 1e-9 m) and their
// warp minimum; pass 2 keeps a triangle for the exact FP64 test when its FP32 distance is within
// eps_d of the activation distance AND (its FP32 barycentrics are inside the band up to eps_b, or its
// FP32 distance is within 2 eps_d of the minimum); survivors are compacted by warp ballot.  Every
// triangle that can form a row in FP64 passes, so the FP64 decisions below see the same candidates
// as a full scan.  The FP64 closest points, the overall minimum, the merge of equal points and the
// ordering by triangle index are spread over the lanes (one survivor per lane).
#include "batch.cuh"
#include "collide_geom.cuh"

namespace accfem {

// Block body: free nodes 4 bx .. 4 bx + 3, one per warp.
__device__ __forceinline__ void collide_body(const Params& p, const Dev& d, int bx) {
  __shared__ int s_list[4][kSurvCap];                 // sorted slots kept for the FP64 test
  __shared__ Surv s_surv[4][kSurvCap];
  __shared__ int s_cand[4][kCandCap];                 // candidate slots (FP32 distance within thr + eps_d)
  __shared__ float s_cd[4][kCandCap];                 // their FP32 distances (negative: near-the-face flag)
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  Ctl* ctl = d.ctl;
  const int f = bx * 4 + wib;
  if (ctl->status != 0 || ctl->converged || f >= ctl->nf) return;
  const int node = ctl->k + 1 + f;
  const double pn[3] = {d.px[node], d.py[node], d.pz[node]};
  const double thr = p.r_o + p.act;
  int lo[3], nc3[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = (int)floor((pn[a] - p.g_rq - p.g_org[a]) / p.g_h);
    int hi = (int)floor((pn[a] + p.g_rq - p.g_org[a]) / p.g_h);
    lo[a] = max(lo[a], 0); hi = min(hi, p.g_dim[a] - 1);
    nc3[a] = max(hi - lo[a] + 1, 0);
  }
  const int ncell = nc3[0] * nc3[1] * nc3[2];
  const float thr32 = (float)(thr + p.eps_d);
  // cell culling: the largest bounding sphere reaches at most g_rq - (r_o + gap) from its centroid;
  // the margin eps_d + 1e-6 m covers the activation margin of the sphere test and the FP32 rounding
  // of the cell-relative coordinates (~1e-9 m)
  const float half_h = (float)(0.5 * p.g_h);
  const float cull_r = (float)(p.g_rq + p.eps_d + 1e-6);
  const float cull_r2 = cull_r * cull_r;
  // Walk of the cells around the node: up to 32 cells at a time, their slot ranges loaded by the
  // lanes and scanned into one index space, so that every round tests 32 slots of any cells (lane
  // j finds its slot's cell by a binary search over the scanned counts) and two rounds' loads are
  // in flight together.  For every 32 slots visit(slot, within, dd, near) is called by the whole
  // warp (within: FP32 distance dd <= r_o + gap + eps_d; near: FP32 barycentrics inside the face
  // band up to eps_b; slots past the end come with within = false).
  auto walk = [&](auto&& visit) {
    for (int c0 = 0; c0 < ncell; c0 += 32) {
      int cs0 = 0, cnt = 0;
      float pcx = 0.f, pcy = 0.f, pcz = 0.f;
      if (c0 + lane < ncell) {
        const int q = c0 + lane;
        const int cx = lo[0] + q % nc3[0];
        const int cy = lo[1] + (q / nc3[0]) % nc3[1];
        const int cz = lo[2] + q / (nc3[0] * nc3[1]);
        pcx = (float)(pn[0] - (p.g_org[0] + (cx + 0.5) * p.g_h));
        pcy = (float)(pn[1] - (p.g_org[1] + (cy + 0.5) * p.g_h));
        pcz = (float)(pn[2] - (p.g_org[2] + (cz + 0.5) * p.g_h));
        // a cell whose box lies farther than cull_r from the node holds no triangle whose bounding
        // sphere reaches the activation distance (its centroid is in the box): its slots are skipped
        const float ex = fmaxf(fabsf(pcx) - half_h, 0.f), ey = fmaxf(fabsf(pcy) - half_h, 0.f),
                    ez = fmaxf(fabsf(pcz) - half_h, 0.f);
        if (ex * ex + ey * ey + ez * ez <= cull_r2) {
          const int cell = (cz * p.g_dim[1] + cy) * p.g_dim[0] + cx;
          cs0 = d.cell_start[cell];
          cnt = d.cell_start[cell + 1] - cs0;
        }
      }
      int incl = cnt;                              // inclusive scan of the slot counts over the lanes
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      const int excl = incl - cnt;
      for (int j0 = 0; j0 < total; j0 += 64) {
        int s[2];
        bool within[2] = {false, false}, near_in[2] = {false, false};
        float dd[2] = {0.f, 0.f}, pc[2][3];
        float4 sp[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int j = j0 + 32 * h + lane;
          const int jc = min(j, total - 1);
          int own = 0;                             // lanes (cells) whose slots all precede jc
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            const int v = __shfl_sync(0xffffffffu, incl, own + step - 1);
            if (v <= jc) own += step;
          }
          s[h] = __shfl_sync(0xffffffffu, cs0, own) + (jc - __shfl_sync(0xffffffffu, excl, own));
          pc[h][0] = __shfl_sync(0xffffffffu, pcx, own);
          pc[h][1] = __shfl_sync(0xffffffffu, pcy, own);
          pc[h][2] = __shfl_sync(0xffffffffu, pcz, own);
          if (j < total) sp[h] = reinterpret_cast<const float4*>(d.sph32)[s[h]];
          if (j >= total) s[h] = -1;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (s[h] >= 0) {
            float dx = pc[h][0] - sp[h].x, dy = pc[h][1] - sp[h].y, dz = pc[h][2] - sp[h].z, rr = thr32 + sp[h].w;
            if (dx * dx + dy * dy + dz * dz <= rr * rr) {
              float va, vb, vc;
              dd[h] = sqrtf(tri_dist2_f32(pc[h], d.tri32 + (size_t)s[h] * 9, va, vb, vc));
              float tol = -((float)kFaceBand + p.eps_b) * (va + vb + vc);
              near_in[h] = (va >= tol) && (vb >= tol) && (vc >= tol);
              within[h] = dd[h] <= thr32;
            }
          }
        }
        visit(s[0], within[0], dd[0], near_in[0]);
        if (j0 + 32 < total) visit(s[1], within[1], dd[1], near_in[1]);
      }
    }
  };
  // ---- pass 1: FP32 candidates (kept in shared memory up to kCandCap) and their minimum distance
  int nca = 0;
  float dmin = 3.0e38f;
  walk([&](int s, bool within, float dd, bool near_in) {
    unsigned mk = __ballot_sync(0xffffffffu, within);
    if (within) {
      dmin = fminf(dmin, dd);
      int pos = nca + __popc(mk & lt_mask);
      if (pos < kCandCap) { s_cand[wib][pos] = s; s_cd[wib][pos] = near_in ? -1.f - dd : dd; }
    }
    nca += __popc(mk);
  });
  __syncwarp();
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dmin = fminf(dmin, __shfl_xor_sync(0xffffffffu, dmin, o));
  const float dmin_keep = dmin + (float)(2.0 * p.eps_d);
  // ---- survivors for the exact test: near the face, or within 2 eps_d of the minimum
  int ns = 0;
  auto survive = [&](bool keep, int slot) {
    unsigned mk = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      int pos = ns + __popc(mk & lt_mask);
      if (pos < kSurvCap) s_list[wib][pos] = slot;
    }
    ns += __popc(mk);
  };
  if (nca <= kCandCap) {
    for (int i0 = 0; i0 < nca; i0 += 32) {
      const int i = i0 + lane;
      bool keep = false;
      if (i < nca) {
        float c = s_cd[wib][i];
        keep = c < 0.f || c <= dmin_keep;
      }
      survive(keep, i < nca ? s_cand[wib][i] : 0);
    }
  } else {
    // more candidates than fit: walk the cells again and filter on the fly
    walk([&](int s, bool within, float dd, bool near_in) { survive(within && (near_in || dd <= dmin_keep), s); });
  }
  __syncwarp();
  if (ns > kSurvCap) {
    if (lane == 0) flag_capacity(ctl, CAP_SURVIVORS);
    return;
  }
  // ---- exact FP64 closest points, one survivor per lane
  for (int i = lane; i < ns; i += 32) {
    int t = d.cell_tri[s_list[wib][i]];
    const int* tv = d.T + 3 * (size_t)t;
    double A[3] = {d.V[3 * tv[0]], d.V[3 * tv[0] + 1], d.V[3 * tv[0] + 2]};
    double Bv[3] = {d.V[3 * tv[1]], d.V[3 * tv[1] + 1], d.V[3 * tv[1] + 2]};
    double Cv[3] = {d.V[3 * tv[2]], d.V[3 * tv[2] + 1], d.V[3 * tv[2] + 2]};
    Surv sv;
    sv.t = t;
    sv.d2 = tri_closest_f64(pn, A, Bv, Cv, sv.c, &sv.interior, &sv.near);
    s_surv[wib][i] = sv;
  }
  __syncwarp();
  // ---- overall closest survivor g: (d2, triangle index) minimum
  double gd = 1.0e300;
  int gt = 0x7fffffff;
  for (int i = lane; i < ns; i += 32) {
    const Surv& sv = s_surv[wib][i];
    if (sv.d2 < gd || (sv.d2 == gd && sv.t < gt)) { gd = sv.d2; gt = sv.t; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double od = __shfl_xor_sync(0xffffffffu, gd, o);
    int ot = __shfl_xor_sync(0xffffffffu, gt, o);
    if (od < gd || (od == gd && ot < gt)) { gd = od; gt = ot; }
  }
  // ---- qualifying survivors: within r_o + gap, and over the face (within the band) or the overall closest
  bool qual[2] = {false, false};
  double dist[2] = {0.0, 0.0};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    int i = lane + 32 * h;
    if (i < ns) {
      const Surv& sv = s_surv[wib][i];
      dist[h] = sqrt(sv.d2);
      qual[h] = (dist[h] <= thr) && (sv.near || sv.t == gt);
    }
  }
  // ---- merge equal closest points (lowest triangle index stays), rank by triangle index
  unsigned qm0 = __ballot_sync(0xffffffffu, qual[0]);
  unsigned qm1 = __ballot_sync(0xffffffffu, qual[1]);
  bool kept[2] = {false, false};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    int i = lane + 32 * h;
    if (!qual[h]) continue;
    const Surv& si = s_surv[wib][i];
    bool dup = false;
    for (int hh = 0; hh < 2 && !dup; ++hh) {
      unsigned mk = hh == 0 ? qm0 : qm1;
      while (mk) {
        int jl = __ffs(mk) - 1;
        mk &= mk - 1;
        int j = jl + 32 * hh;
        const Surv& sj = s_surv[wib][j];
        if (sj.t >= si.t) continue;
        double dx = sj.c[0] - si.c[0], dy = sj.c[1] - si.c[1], dz = sj.c[2] - si.c[2];
        // |c_j - c_i| <= 1e-12 m, compared squared (points of one wall feature differ by ~1e-17 m,
        // distinct ones by micrometres, so no decision sits near the threshold)
        if (dx * dx + dy * dy + dz * dz <= 1e-24) { dup = true; break; }
      }
    }
    kept[h] = !dup;
  }
  unsigned km0 = __ballot_sync(0xffffffffu, kept[0]);
  unsigned km1 = __ballot_sync(0xffffffffu, kept[1]);
  const int nc = __popc(km0) + __popc(km1);
  if (nc > kCpn) {
    if (lane == 0) flag_capacity(ctl, CAP_NODE_ROWS);
    return;
  }
  int* ctri = d.con_tri + (size_t)f * kListCap;
  double* cpt = d.con_pt + (size_t)f * kListCap * 3;
  double* cn = d.con_n + (size_t)f * kListCap * 3;
  double* cg = d.con_gap + (size_t)f * kListCap;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if (!kept[h]) continue;
    const Surv& sv = s_surv[wib][lane + 32 * h];
    int rank = 0;
    for (int hh = 0; hh < 2; ++hh) {
      unsigned mk = hh == 0 ? km0 : km1;
      while (mk) {
        int jl = __ffs(mk) - 1;
        mk &= mk - 1;
        if (s_surv[wib][jl + 32 * hh].t < sv.t) ++rank;
      }
    }
    const double* nf = d.nface + 3 * (size_t)sv.t;
    double n[3];
    double cmp[3] = {sv.c[0] - pn[0], sv.c[1] - pn[1], sv.c[2] - pn[2]};
    if (sv.interior || dist[h] < 1e-12) { n[0] = nf[0]; n[1] = nf[1]; n[2] = nf[2]; }
    else {
      double sgn = (dot3(nf, cmp) > 0.0) ? 1.0 : -1.0;
      double id = sgn / dist[h];
      n[0] = cmp[0] * id; n[1] = cmp[1] * id; n[2] = cmp[2] * id;
    }
    ctri[rank] = sv.t;
    cpt[3 * rank] = sv.c[0]; cpt[3 * rank + 1] = sv.c[1]; cpt[3 * rank + 2] = sv.c[2];
    cn[3 * rank] = n[0]; cn[3 * rank + 1] = n[1]; cn[3 * rank + 2] = n[2];
    cg[rank] = dot3(n, sv.c) - dot3(n, pn) - p.r_o;
  }
  if (lane == 0) d.ncon[f] = nc;
}

__global__ void __launch_bounds__(128) collide_kernel(Params p, Dev d) {
  pdl_enter();
  collide_body(p, d, blockIdx.x);
}

// Node rows of the batch's members with the node contact model (segment members: segment.cu).
__global__ void __launch_bounds__(128) collide_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan) {
  for_units(tab, plan, PH_COLL, [](const Inst& in, int bx, int) {
    if (in.p.contact_model == kContactNode) collide_body(in.p, in.d, bx);
  });
}

}  // namespace accfem
