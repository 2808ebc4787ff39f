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

__device__ __forceinline__ double dist3(const double* a, const double* b) {
  const double d[3] = {a[0] - b[0], a[1] - b[1], a[2] - b[2]};
  return sqrt(dot3(d, d));
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

// Closest point of triangle (a, b, c) to p by its plain definition; returns |p - w|.
__device__ double tri_point(const double* p, const double* a, const double* b, const double* c, const double* n,
                            double* w) {
  double proj[3], v, ww;
  project(p, a, n, proj);
  bary2(proj, a, b, c, &v, &ww);
  if (v >= 0.0 && ww >= 0.0 && v + ww <= 1.0) {
    w[0] = proj[0]; w[1] = proj[1]; w[2] = proj[2];
    return dist3(p, proj);
  }
  const double* E[3][2] = {{a, b}, {b, c}, {c, a}};
  double bd = 1.0e300;
  for (int k = 0; k < 3; ++k) {
    double q[3];
    seg_point(E[k][0], E[k][1], p, q);
    const double d = dist3(p, q);
    if (d < bd) { bd = d; w[0] = q[0]; w[1] = q[1]; w[2] = q[2]; }
  }
  return bd;
}

// Closest points of segments p0 p1 and q0 q1: parameters (s, t), points x, y; returns |x - y|.
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
    const double d = dist3(x, y);
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
    *interior = (v >= 0.0 && ww >= 0.0 && v + ww <= 1.0 && dist3(proj, w) <= 1e-15 * sc) ? 1 : 0;
  }
  return best;
}

// A chord within r_o + gap of a wall lies near more triangles than a node does: up to kSegSurvCap of
// them get the exact test (4 warps of a block: 41 KB of shared memory).
constexpr int kSegSurvCap = 144;

struct SegSurv {
  int t;
  short interior, near;
  double d, s, q[3], w[3];
};

}  // namespace seg

using namespace seg;

// Block body: free elements 4 bx .. 4 bx + 3, one per warp (element k + f joins nodes k + f and
// k + 1 + f).  Candidates from the grid cells around the chord; a triangle whose bounding sphere
// stays beyond the activation distance is skipped, every other one gets the exact FP64 test.
__device__ __forceinline__ void collide_segment_body(const Params& p, const Dev& d, int bx) {
  __shared__ SegSurv s_surv[4][kSegSurvCap];
  __shared__ int s_ns[4];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  Ctl* ctl = d.ctl;
  const int f = bx * 4 + wib;
  if (ctl->status != 0 || ctl->converged || f >= ctl->nf) return;
  const int na = ctl->k + f, nb = na + 1;
  const double p0[3] = {d.px[na], d.py[na], d.pz[na]};
  const double p1[3] = {d.px[nb], d.py[nb], d.pz[nb]};
  const double thr = p.r_o + p.act;
  if (lane == 0) s_ns[wib] = 0;
  __syncwarp();
  int lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = max((int)floor((fmin(p0[a], p1[a]) - p.g_rq - p.g_org[a]) / p.g_h), 0);
    hi[a] = min((int)floor((fmax(p0[a], p1[a]) + p.g_rq - p.g_org[a]) / p.g_h), p.g_dim[a] - 1);
  }
  for (int cz = lo[2]; cz <= hi[2]; ++cz)
    for (int cy = lo[1]; cy <= hi[1]; ++cy)
      for (int cx = lo[0]; cx <= hi[0]; ++cx) {
        const int cell = (cz * p.g_dim[1] + cy) * p.g_dim[0] + cx;
        const int s0 = d.cell_start[cell], s1 = d.cell_start[cell + 1];
        for (int sl = s0 + lane; sl < s1; sl += 32) {
          const int t = d.cell_tri[sl];
          const int* tv = d.T + 3 * (size_t)t;
          const double A[3] = {d.V[3 * tv[0]], d.V[3 * tv[0] + 1], d.V[3 * tv[0] + 2]};
          const double B[3] = {d.V[3 * tv[1]], d.V[3 * tv[1] + 1], d.V[3 * tv[1] + 2]};
          const double C[3] = {d.V[3 * tv[2]], d.V[3 * tv[2] + 1], d.V[3 * tv[2] + 2]};
          // bounding sphere of the triangle (centroid, farthest vertex) against the chord
          const double cen[3] = {(A[0] + B[0] + C[0]) / 3.0, (A[1] + B[1] + C[1]) / 3.0, (A[2] + B[2] + C[2]) / 3.0};
          const double rad = fmax(dist3(cen, A), fmax(dist3(cen, B), dist3(cen, C)));
          double qc[3];
          seg_point(p0, p1, cen, qc);
          if (dist3(qc, cen) - rad > thr * (1.0 + 1e-12) + 1e-12) continue;
          const double* nf = d.nface + 3 * (size_t)t;
          SegSurv sv;
          sv.t = t;
          int inside = 0;
          sv.d = seg_tri(p0, p1, A, B, C, nf, &sv.s, sv.q, sv.w, &inside);
          sv.interior = (short)inside;
          if (!(sv.d <= thr)) continue;
          double pr[3], v, ww;
          project(sv.q, A, nf, pr);
          bary2(pr, A, B, C, &v, &ww);
          sv.near = (v >= -kFaceBand && ww >= -kFaceBand && 1.0 - v - ww >= -kFaceBand) ? 1 : 0;
          const int slot = atomicAdd(&s_ns[wib], 1);
          if (slot < kSegSurvCap) s_surv[wib][slot] = sv;
        }
      }
  __syncwarp();
  const int ns = s_ns[wib];
  if (lane != 0) return;
  if (ns > kSegSurvCap) {
    d.ncon[f] = 0;
    flag_capacity(ctl, CAP_SURVIVORS);
    return;
  }
  // the element's closest triangle (smallest distance, lowest index on ties)
  int g = -1;
  for (int i = 0; i < ns; ++i) {
    const SegSurv& sv = s_surv[wib][i];
    if (g < 0 || sv.d < s_surv[wib][g].d || (sv.d == s_surv[wib][g].d && sv.t < s_surv[wib][g].t)) g = i;
  }
  int ord[kSegSurvCap];
  for (int i = 0; i < ns; ++i) {                   // by triangle index
    int j = i;
    while (j > 0 && s_surv[wib][ord[j - 1]].t > s_surv[wib][i].t) { ord[j] = ord[j - 1]; --j; }
    ord[j] = i;
  }
  int nc = 0;
  int* ctri = d.con_tri + (size_t)f * kListCap;
  double* cpt = d.con_pt + (size_t)f * kListCap * 3;
  double* cn = d.con_n + (size_t)f * kListCap * 3;
  double* cg = d.con_gap + (size_t)f * kListCap;
  double* cs = d.con_s + (size_t)f * kListCap;
  double kq[kSegCpn][3];
  for (int oi = 0; oi < ns; ++oi) {
    const SegSurv& sv = s_surv[wib][ord[oi]];
    if (!(sv.near || ord[oi] == g)) continue;
    bool dup = false;
    for (int r = 0; r < nc && !dup; ++r)
      dup = dist3(cpt + 3 * r, sv.w) <= 1e-12 && dist3(kq[r], sv.q) <= 1e-12;
    if (dup) continue;
    if (nc >= kSegCpn) { flag_capacity(ctl, CAP_NODE_ROWS); break; }
    const double* nf = d.nface + 3 * (size_t)sv.t;
    double nv[3];
    if (sv.interior || sv.d < 1e-12) { nv[0] = nf[0]; nv[1] = nf[1]; nv[2] = nf[2]; }
    else {
      const double id = 1.0 / sv.d;
      nv[0] = (sv.w[0] - sv.q[0]) * id; nv[1] = (sv.w[1] - sv.q[1]) * id; nv[2] = (sv.w[2] - sv.q[2]) * id;
      if (dot3(nv, nf) < 0.0) { nv[0] = -nv[0]; nv[1] = -nv[1]; nv[2] = -nv[2]; }
    }
    ctri[nc] = sv.t;
    for (int i = 0; i < 3; ++i) { cpt[3 * nc + i] = sv.w[i]; cn[3 * nc + i] = nv[i]; kq[nc][i] = sv.q[i]; }
    cg[nc] = dot3(nv, sv.w) - dot3(nv, sv.q) - p.r_o;
    cs[nc] = sv.s;
    ++nc;
  }
  d.ncon[f] = nc;
}

__global__ void __launch_bounds__(128) collide_segment_kernel(Params p, Dev d) {
  pdl_enter();
  collide_segment_body(p, d, blockIdx.x);
}

// Segment rows of the batch's members with the segment contact model (launched beside collide_batch
// when the batch has such members).
__global__ void __launch_bounds__(128) collide_segment_batch(const Inst* __restrict__ tab, const Plan* __restrict__ plan) {
  for_units(tab, plan, PH_COLL, [](const Inst& in, int bx, int) {
    if (in.p.contact_model == kContactSegment) collide_segment_body(in.p, in.d, bx);
  });
}

}  // namespace accfem
