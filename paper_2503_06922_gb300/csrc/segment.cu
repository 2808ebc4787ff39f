// Segment contacts (Eq. 3-7 at any point of an element): the constraint rows of element chords
// against the lumen triangles.  A contact point lies at chord fraction s of element e (nodes e and
// e + 1); its displacement is interpolated from the two nodal translations by N(xi) of Eq. 4-6 in
// the element frame (the weights are formed at compaction, btd.cu).
//
// Row rule per element (the same as the node rule, with the chord for the node): with (q_t, w_t)
// the closest points of the chord and triangle t, d_t = |w_t - q_t| and g the triangle of smallest
// d_t (lowest index on ties), (element, t) is a row when d_t <= r_o + activation gap and either t is
// g or the plane projection of q_t lies inside t enlarged by the barycentric margin kFaceBand.  The
// normal is the face normal for a wall point inside the face (or d_t < 1e-12), else along w_t - q_t,
// flipped outward.  Rows of one element with the same pair of closest points (1e-12 m) are merged,
// keeping the lowest index; a row at a shared node (s = 0 here, s = 1 on the element before, the
// same wall point) is kept once, on the lower element (at compaction).
//
// Closest points of a segment and a triangle, by the plain case split: if the segment crosses the
// triangle, the crossing point at distance 0; otherwise the nearer of a segment endpoint against
// the triangle (closest point on a triangle: plane projection when inside, else the nearest
// clamped edge projection) and the segment against each triangle edge (closest points of two
// segments: the interior stationary point of |p0 + s d1 - q0 - t d2|^2 on the unit square when it
// lies there, else the best of the four edges of the square, each a clamped 1-D minimum).
#include "batch.cuh"
#include "collide_geom.cuh"

namespace accfem {

namespace seg {

__device__ __forceinline__ void sub3(const double* a, const double* b, double* c) {
  c[0] = a[0] - b[0]; c[1] = a[1] - b[1]; c[2] = a[2] - b[2];
}

// Squared distance: the candidates below are compared by it, so a test takes one square root.
__device__ __forceinline__ double dist2(const double* a, const double* b) {
  const double d[3] = {a[0] - b[0], a[1] - b[1], a[2] - b[2]};
  return dot3(d, d);
}

// Barycentric coordinates (v, w) of the point x in the plane of (a, b, c): x - a = v (b - a) + w (c - a).
__device__ __forceinline__ void bary2(const double* x, const double* a, const double* b, const double* c, double* v,
                                      double* w) {
  double ab[3], ac[3], ax[3];
  sub3(b, a, ab); sub3(c, a, ac); sub3(x, a, ax);
  const double m00 = dot3(ab, ab), m01 = dot3(ab, ac), m11 = dot3(ac, ac);
  const double r0 = dot3(ab, ax), r1 = dot3(ac, ax);
  const double det = m00 * m11 - m01 * m01;
  *v = (m11 * r0 - m01 * r1) / det;
  *w = (m00 * r1 - m01 * r0) / det;
}

// Plane projection of x onto the triangle's plane (unit normal n through a).
__device__ __forceinline__ void project(const double* x, const double* a, const double* n, double* out) {
  double ax[3];
  sub3(x, a, ax);
  const double h = dot3(n, ax);
  out[0] = x[0] - h * n[0]; out[1] = x[1] - h * n[1]; out[2] = x[2] - h * n[2];
}

// Closest point of segment s0 s1 to p: the clamped projection.
__device__ __forceinline__ void seg_point(const double* s0, const double* s1, const double* p, double* q) {
  double e[3], sp[3];
  sub3(s1, s0, e); sub3(p, s0, sp);
  double t = dot3(sp, e) / dot3(e, e);
  t = fmin(1.0, fmax(0.0, t));
  q[0] = s0[0] + t * e[0]; q[1] = s0[1] + t * e[1]; q[2] = s0[2] + t * e[2];
}

// Closest point of triangle (a, b, c) to p by its plain definition; returns |p - w|^2.
__device__ double tri_point(const double* p, const double* a, const double* b, const double* c, const double* n,
                            double* w) {
  double proj[3], v, ww;
  project(p, a, n, proj);
  bary2(proj, a, b, c, &v, &ww);
  if (v >= 0.0 && ww >= 0.0 && v + ww <= 1.0) {
    w[0] = proj[0]; w[1] = proj[1]; w[2] = proj[2];
    return dist2(p, proj);
  }
  const double* E[3][2] = {{a, b}, {b, c}, {c, a}};
  double bd = 1.0e300;
  for (int k = 0; k < 3; ++k) {
    double q[3];
    seg_point(E[k][0], E[k][1], p, q);
    const double d = dist2(p, q);
    if (d < bd) { bd = d; w[0] = q[0]; w[1] = q[1]; w[2] = q[2]; }
  }
  return bd;
}

// Closest points of segments p0 p1 and q0 q1: parameters (s, t), points x, y; returns |x - y|^2.
__device__ double seg_seg(const double* p0, const double* p1, const double* q0, const double* q1, double* s_out,
                          double* x_out, double* y_out) {
  double d1[3], d2[3], r[3];
  sub3(p1, p0, d1); sub3(q1, q0, d2); sub3(p0, q0, r);
  const double a = dot3(d1, d1), e = dot3(d2, d2), b = dot3(d1, d2), c = dot3(d1, r), f = dot3(d2, r);
  double cs[5], ct[5];
  int nc = 0;
  const double den = a * e - b * b;
  if (den > 1e-30 * a * e) {
    const double s = (b * f - c * e) / den, t = (a * f - b * c) / den;
    if (s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0) { cs[nc] = s; ct[nc] = t; ++nc; }
  }
  for (int k = 0; k < 2; ++k) {                    // edges s = 0, 1
    const double s = (double)k;
    cs[nc] = s;
    ct[nc] = e > 0.0 ? fmin(1.0, fmax(0.0, (b * s + f) / e)) : 0.0;
    ++nc;
  }
  for (int k = 0; k < 2; ++k) {                    // edges t = 0, 1
    const double t = (double)k;
    cs[nc] = a > 0.0 ? fmin(1.0, fmax(0.0, (b * t - c) / a)) : 0.0;
    ct[nc] = t;
    ++nc;
  }
  double best = 1.0e300;
  for (int k = 0; k < nc; ++k) {
    const double x[3] = {p0[0] + cs[k] * d1[0], p0[1] + cs[k] * d1[1], p0[2] + cs[k] * d1[2]};
    const double y[3] = {q0[0] + ct[k] * d2[0], q0[1] + ct[k] * d2[1], q0[2] + ct[k] * d2[2]};
    const double d = dist2(x, y);
    if (d < best) {
      best = d;
      *s_out = cs[k];
      for (int i = 0; i < 3; ++i) { x_out[i] = x[i]; y_out[i] = y[i]; }
    }
  }
  return best;
}

// Closest points of the segment p0 p1 and triangle (a, b, c) with unit normal n: chord fraction s,
// segment point q, wall point w, distance, and whether w is inside the face.
__device__ double seg_tri(const double* p0, const double* p1, const double* a, const double* b, const double* c,
                          const double* n, double* s_out, double* q, double* w, int* interior) {
  double ap0[3], ap1[3];
  sub3(p0, a, ap0); sub3(p1, a, ap1);
  const double h0 = dot3(n, ap0), h1 = dot3(n, ap1);
  if (h0 * h1 < 0.0) {
    const double s = h0 / (h0 - h1);
    const double x[3] = {p0[0] + s * (p1[0] - p0[0]), p0[1] + s * (p1[1] - p0[1]), p0[2] + s * (p1[2] - p0[2])};
    double xp[3], v, ww;
    project(x, a, n, xp);
    bary2(xp, a, b, c, &v, &ww);
    if (v >= 0.0 && ww >= 0.0 && v + ww <= 1.0) {
      *s_out = s;
      for (int i = 0; i < 3; ++i) { q[i] = x[i]; w[i] = xp[i]; }
      *interior = 1;
      return 0.0;
    }
  }
  double best = 1.0e300;
  int endpoint = 1;
  for (int k = 0; k < 2; ++k) {
    const double* pt = k == 0 ? p0 : p1;
    double wt[3];
    const double d = tri_point(pt, a, b, c, n, wt);
    if (d < best) {
      best = d;
      *s_out = (double)k;
      for (int i = 0; i < 3; ++i) { q[i] = pt[i]; w[i] = wt[i]; }
    }
  }
  const double* E[3][2] = {{a, b}, {b, c}, {c, a}};
  for (int k = 0; k < 3; ++k) {
    double s, x[3], y[3];
    const double d = seg_seg(p0, p1, E[k][0], E[k][1], &s, x, y);
    if (d < best) {
      best = d;
      endpoint = 0;
      *s_out = s;
      for (int i = 0; i < 3; ++i) { q[i] = x[i]; w[i] = y[i]; }
    }
  }
  *interior = 0;
  if (endpoint) {                                  // inside when the projection is the wall point
    double proj[3], v, ww;
    project(q, a, n, proj);
    bary2(proj, a, b, c, &v, &ww);
    const double sc = fmax(1.0, fmax(fabs(w[0]), fmax(fabs(w[1]), fabs(w[2]))));
    *interior = (v >= 0.0 && ww >= 0.0 && v + ww <= 1.0 && dist2(proj, w) <= (1e-15 * sc) * (1e-15 * sc)) ? 1 : 0;
  }
  return sqrt(best);
}

// A chord within r_o + gap of a wall lies near more triangles than a node does: up to kSegSurvCap of
// them get the exact test.
constexpr int kSegSurvCap = 144;

struct SegSurv {
  int t;
  short interior, near;
  double d, s, q[3], w[3];
};

}  // namespace seg

using namespace seg;

// Block body: free element f (element k + f, joining nodes k + f and k + 1 + f), four warps sharing
// its candidate slots and survivor list.  Candidates from the grid cells around the chord; a triangle whose FP32 bounding
// sphere, or whose plane and edge slabs, stay beyond the activation distance (+ eps_d) is
// skipped, every other one gets the exact FP64 test.
__device__ __forceinline__ void collide_segment_body(const Params& p, const Dev& d, int f) {
  __shared__ SegSurv s_surv[kSegSurvCap];
  __shared__ int s_queue[4][64];                   // slots that passed the FP32 bounds, per warp
  __shared__ int s_ns;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  Ctl* ctl = d.ctl;
  if (ctl->status != 0 || ctl->converged || f >= ctl->nf) return;
  const int na = ctl->k + f, nb = na + 1;
  const double p0[3] = {d.px[na], d.py[na], d.pz[na]};
  const double p1[3] = {d.px[nb], d.py[nb], d.pz[nb]};
  const double thr = p.r_o + p.act;
  if (threadIdx.x == 0) s_ns = 0;
  __syncthreads();
  int lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = max((int)floor((fmin(p0[a], p1[a]) - p.g_rq - p.g_org[a]) / p.g_h), 0);
    hi[a] = min((int)floor((fmax(p0[a], p1[a]) + p.g_rq - p.g_org[a]) / p.g_h), p.g_dim[a] - 1);
  }
  const float thr32 = (float)(thr + p.eps_d);
  const unsigned lt_mask = (1u << lane) - 1u;
  // Exact FP64 test of the queued slots q[0 .. n) (n <= 32), one per lane; survivors within r_o +
  // gap go to the warp's list.  Queuing the slots that pass the FP32 bounds first keeps all lanes
  // of a round of the (long) exact test busy.
  int* q = s_queue[wib];
  auto exact = [&](int n) {
    if (lane < n) {
      const int t = d.cell_tri[q[lane]];
      const double* nf = d.nface + 3 * (size_t)t;
      const int* tv = d.T + 3 * (size_t)t;
      const double A[3] = {d.V[3 * tv[0]], d.V[3 * tv[0] + 1], d.V[3 * tv[0] + 2]};
      const double B[3] = {d.V[3 * tv[1]], d.V[3 * tv[1] + 1], d.V[3 * tv[1] + 2]};
      const double C[3] = {d.V[3 * tv[2]], d.V[3 * tv[2] + 1], d.V[3 * tv[2] + 2]};
      SegSurv sv;
      sv.t = t;
      int inside = 0;
      sv.d = seg_tri(p0, p1, A, B, C, nf, &sv.s, sv.q, sv.w, &inside);
      sv.interior = (short)inside;
      if (sv.d <= thr) {
        double pr[3], v, ww;
        project(sv.q, A, nf, pr);
        bary2(pr, A, B, C, &v, &ww);
        sv.near = (v >= -kFaceBand && ww >= -kFaceBand && 1.0 - v - ww >= -kFaceBand) ? 1 : 0;
        const int slot = atomicAdd(&s_ns, 1);
        if (slot < kSegSurvCap) s_surv[slot] = sv;
      }
    }
    __syncwarp();
  };
  int nc3[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) nc3[a] = max(hi[a] - lo[a] + 1, 0);
  const int ncell = nc3[0] * nc3[1] * nc3[2];
  const float e0 = (float)(p1[0] - p0[0]), e1 = (float)(p1[1] - p0[1]), e2 = (float)(p1[2] - p0[2]);
  const float ee = e0 * e0 + e1 * e1 + e2 * e2;
  int nq = 0;                                      // queued slots (the same in every lane)
  // Walk of the cells around the chord, 32 cells at a time: lane l loads cell c0 + l's slot range
  // and the chord's start relative to that cell's centre (the frame of the FP32 triangle data: FP32
  // coordinates of a few mm, errors of a few 1e-9 m, far inside the margin eps_d); the ranges are
  // scanned into one index space, and every round tests 32 slots of any of these cells (the lane of a
  // slot's cell found by a binary search over the scanned counts).
  for (int c0 = 0; c0 < ncell; c0 += 32) {
    int cs0 = 0, cnt = 0;
    float ra0 = 0.f, ra1 = 0.f, ra2 = 0.f;
    if (c0 + lane < ncell) {
      const int qc = c0 + lane;
      const int cx = lo[0] + qc % nc3[0], cy = lo[1] + (qc / nc3[0]) % nc3[1], cz = lo[2] + qc / (nc3[0] * nc3[1]);
      const int cell = (cz * p.g_dim[1] + cy) * p.g_dim[0] + cx;
      cs0 = d.cell_start[cell];
      cnt = d.cell_start[cell + 1] - cs0;
      ra0 = (float)(p0[0] - (p.g_org[0] + (cx + 0.5) * p.g_h));
      ra1 = (float)(p0[1] - (p.g_org[1] + (cy + 0.5) * p.g_h));
      ra2 = (float)(p0[2] - (p.g_org[2] + (cz + 0.5) * p.g_h));
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    const int excl = incl - cnt;
    for (int j0 = 32 * wib; j0 < total; j0 += 128) {   // the four warps share the slots
      const int j = j0 + lane;
      const int jc = min(j, total - 1);
      int own = 0;                                 // lanes (cells) whose slots all precede jc
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int v = __shfl_sync(0xffffffffu, incl, own + step - 1);
        if (v <= jc) own += step;
      }
      const int sl = __shfl_sync(0xffffffffu, cs0, own) + (jc - __shfl_sync(0xffffffffu, excl, own));
      const float ca0 = __shfl_sync(0xffffffffu, ra0, own), ca1 = __shfl_sync(0xffffffffu, ra1, own),
                  ca2 = __shfl_sync(0xffffffffu, ra2, own);
      // FP32 lower bounds of the chord-triangle distance, each only skipping a triangle that is
      // farther than r_o + gap + eps_d: the bounding sphere, then the plane and edge slabs
      bool pass = false;
      if (j < total) {
        const float4 sp = reinterpret_cast<const float4*>(d.sph32)[sl];
        float tt = ee > 0.f ? ((sp.x - ca0) * e0 + (sp.y - ca1) * e1 + (sp.z - ca2) * e2) / ee : 0.f;
        tt = fminf(1.f, fmaxf(0.f, tt));
        const float qx = ca0 + tt * e0 - sp.x, qy = ca1 + tt * e1 - sp.y, qz = ca2 + tt * e2 - sp.z;
        const float rr = thr32 + sp.w;
        if (qx * qx + qy * qy + qz * qz <= rr * rr) {
          const double* nf = d.nface + 3 * (size_t)d.cell_tri[sl];
          const float n[3] = {(float)nf[0], (float)nf[1], (float)nf[2]};
          const float* v = d.tri32 + (size_t)sl * 9;
          const float pa[3] = {ca0, ca1, ca2}, pb[3] = {ca0 + e0, ca1 + e1, ca2 + e2};
          // height over the plane (0 when the chord crosses it) and, beside it, the distance
          // outside the triangle's edges: the slab of edge k is the half-space through the edge
          // with the in-plane outward normal m_k, and the triangle lies in all three; both are
          // linear along the chord, so their minima are at an endpoint.  A point of the chord
          // is at least sqrt(h^2 + e^2) from the triangle, h and e being orthogonal parts.
          float h0 = 0.f, h1 = 0.f;
          for (int c = 0; c < 3; ++c) { h0 += n[c] * (pa[c] - v[c]); h1 += n[c] * (pb[c] - v[c]); }
          const float hmin = h0 * h1 > 0.f ? fminf(fabsf(h0), fabsf(h1)) : 0.f;
          float emax = 0.f;
#pragma unroll
          for (int k = 0; k < 3; ++k) {
            const float* vi = v + 3 * k;
            const float* vj = v + 3 * ((k + 1) % 3);
            const float* vk = v + 3 * ((k + 2) % 3);
            const float ed[3] = {vj[0] - vi[0], vj[1] - vi[1], vj[2] - vi[2]};
            float m[3] = {ed[1] * n[2] - ed[2] * n[1], ed[2] * n[0] - ed[0] * n[2], ed[0] * n[1] - ed[1] * n[0]};
            const float mm = m[0] * m[0] + m[1] * m[1] + m[2] * m[2];
            if (!(mm > 0.f)) continue;                // degenerate edge: no bound from it
            const float im = rsqrtf(mm);
            float sk = 0.f;
            for (int c = 0; c < 3; ++c) { m[c] *= im; sk += m[c] * (vk[c] - vi[c]); }
            if (!(fabsf(sk) > 1e-9f)) continue;      // no clear inside (a sliver): no bound
            const float sg = sk > 0.f ? -1.f : 1.f;   // outward: away from the third vertex
            float s0 = 0.f, s1 = 0.f;
            for (int c = 0; c < 3; ++c) { s0 += m[c] * (pa[c] - vi[c]); s1 += m[c] * (pb[c] - vi[c]); }
            emax = fmaxf(emax, fminf(sg * s0, sg * s1));
          }
          pass = hmin * hmin + emax * emax <= thr32 * thr32;
        }
      }
      const unsigned mk = __ballot_sync(0xffffffffu, pass);
      if (pass) q[nq + __popc(mk & lt_mask)] = sl;
      nq += __popc(mk);
      __syncwarp();
      if (nq >= 32) {                              // a full round; the rest (< 32) moves to the front
        exact(32);
        const int rest = nq - 32;
        const int mv = lane < rest ? q[32 + lane] : 0;
        __syncwarp();
        if (lane < rest) q[lane] = mv;
        __syncwarp();
        nq = rest;
      }
    }
  }
  if (nq > 0) exact(nq);
  __syncthreads();
  if (wib != 0) return;                            // warp 0 selects the rows
  const int ns = s_ns;
  if (ns > kSegSurvCap) {
    if (lane == 0) {
      d.ncon[f] = 0;
      flag_capacity(ctl, CAP_SURVIVORS);
    }
    return;
  }
  const SegSurv* sv = s_surv;
  // the element's closest triangle (smallest distance, lowest index on ties): warp argmin
  double gd = 1.0e300;
  int gt = 0x7fffffff, gi = -1;
  for (int i = lane; i < ns; i += 32)
    if (sv[i].d < gd || (sv[i].d == gd && sv[i].t < gt)) { gd = sv[i].d; gt = sv[i].t; gi = i; }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double od = __shfl_xor_sync(0xffffffffu, gd, o);
    const int ot = __shfl_xor_sync(0xffffffffu, gt, o), oi = __shfl_xor_sync(0xffffffffu, gi, o);
    if (od < gd || (od == gd && ot < gt)) { gd = od; gt = ot; gi = oi; }
  }
  // rank of each survivor by triangle index (rows in triangle order; a triangle is in one cell, so
  // the indices differ); lane l keeps the ranks of survivors l, l + 32, ...
  constexpr int kPer = (kSegSurvCap + 31) / 32;
  int rk[kPer];
#pragma unroll
  for (int h = 0; h < kPer; ++h) {
    const int i = lane + 32 * h;
    rk[h] = -1;
    if (i < ns) {
      int r = 0;
      for (int j = 0; j < ns; ++j) r += sv[j].t < sv[i].t ? 1 : 0;
      rk[h] = r;
    }
  }
  // rows in triangle order; lane r keeps accepted row r's wall and chord points for the merge test
  int* ctri = d.con_tri + (size_t)f * kListCap;
  double* cpt = d.con_pt + (size_t)f * kListCap * 3;
  double* cn = d.con_n + (size_t)f * kListCap * 3;
  double* cg = d.con_gap + (size_t)f * kListCap;
  double* cs = d.con_s + (size_t)f * kListCap;
  double kw[3] = {0.0, 0.0, 0.0}, kq[3] = {0.0, 0.0, 0.0};
  int nc = 0;
  for (int oi = 0; oi < ns; ++oi) {
    int own = -1;
#pragma unroll
    for (int h = 0; h < kPer; ++h)
      if (rk[h] == oi) own = lane + 32 * h;
    const unsigned mk = __ballot_sync(0xffffffffu, own >= 0);
    const int i = __shfl_sync(0xffffffffu, own, __ffs(mk) - 1);
    const SegSurv& c = sv[i];
    if (!(c.near || i == gi)) continue;
    const bool dup = lane < nc && dist2(kw, c.w) <= 1e-24 && dist2(kq, c.q) <= 1e-24;
    if (__any_sync(0xffffffffu, dup)) continue;
    if (nc >= kSegCpn) {
      if (lane == 0) flag_capacity(ctl, CAP_NODE_ROWS);
      break;
    }
    if (lane == nc) {
      const double* nf = d.nface + 3 * (size_t)c.t;
      double nv[3];
      if (c.interior || c.d < 1e-12) { nv[0] = nf[0]; nv[1] = nf[1]; nv[2] = nf[2]; }
      else {
        const double id = 1.0 / c.d;
        nv[0] = (c.w[0] - c.q[0]) * id; nv[1] = (c.w[1] - c.q[1]) * id; nv[2] = (c.w[2] - c.q[2]) * id;
        if (dot3(nv, nf) < 0.0) { nv[0] = -nv[0]; nv[1] = -nv[1]; nv[2] = -nv[2]; }
      }
      ctri[nc] = c.t;
      for (int k = 0; k < 3; ++k) { cpt[3 * nc + k] = c.w[k]; cn[3 * nc + k] = nv[k]; kw[k] = c.w[k]; kq[k] = c.q[k]; }
      cg[nc] = dot3(nv, c.w) - dot3(nv, c.q) - p.r_o;
      cs[nc] = c.s;
    }
    ++nc;
  }
  if (lane == 0) d.ncon[f] = nc;
}

__global__ void __launch_bounds__(128) collide_segment_kernel(Params p, Dev d) {
  pdl_enter();
  collide_segment_body(p, d, blockIdx.x);
}

// Segment rows of the batch's members with the segment contact model (launched beside collide_batch
// when the batch has such members): a unit of the collision phase is four elements, taken in turn.
__global__ void __launch_bounds__(128) collide_segment_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan) {
  for_units(tab, plan, PH_COLL, [](const Inst& in, int bx, int) {
    if (in.p.contact_model != kContactSegment) return;
    for (int e = 0; e < 4; ++e) {
      collide_segment_body(in.p, in.d, 4 * bx + e);
      __syncthreads();
    }
  });
}

}  // namespace accfem
