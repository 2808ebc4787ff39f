// Internal definitions shared by the CUDA translation units of the Acc-FEM hot path.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace accfem {

constexpr int kMaxCables = 8;
constexpr int kCpn = 16;           // constraint rows per node (wall features the node lies over)
constexpr int kSegCpn = 32;        // constraint rows per element in the segment model (a chord lies over more)
constexpr int kListCap = 32;       // slots of a per-owner constraint list (>= kCpn, kSegCpn)
constexpr int kSurvCap = 64;       // FP64 candidates per node after the FP32 prefilter
constexpr int kCandCap = 256;      // candidates per node kept in shared memory (more: a second cell walk)
constexpr int kElemStride = 96;    // doubles per element record: 78 K (upper) + 12 F + pad
constexpr int kWarpsPerElemBlock = 2;
constexpr int kRhsSplit = 4;       // blocks per node that share the RHS columns (chunks of 32)
constexpr int kBwdSplit = 8;       // back substitution: blocks per node (chunks of 16 columns, 96 threads)
constexpr int kMaxWorking = 512;   // rows of the contact working set (RHS columns, LCP size)
constexpr int kPrecisionFP64 = 0, kPrecisionMixed = 1;
// Anderson acceleration of the Newton iteration: previous iterates used, and the largest
// sum |gamma_j| of an accepted accelerated step (the same values are used by the CPU oracle).
constexpr int kAccelDepth = 3;
constexpr int kAccelSlots = kAccelDepth + 1;   // ring of held iterates: the slot written in iteration k is
                                              // none of the k - 1 .. k - kAccelDepth that are read then
constexpr double kAccelGammaMax = 10.0;
constexpr int kAccelParts = 10;    // per step block: G (6 upper entries) and b (3) of the least squares, sum |du|^2
// Iterations of a solve that may take Anderson steps; later ones (and the FP32 tangent's) fall back to
// the 1-D secant over-relaxation of a slow monotone mode.
constexpr int kAccelIters = 100;
constexpr int kLcpActiveSet = 0, kLcpAdmm = 1, kLcpPrimalAdmm = 2;
// The single-instance contact kernel is launched with this many bytes of dynamic shared memory: the
// ADMM contact solver inverts its FP32 matrix there for working sets of up to kAdmmSmemRows rows, the
// active-set LCP keeps W there for up to 135 rows (larger ones in global memory).
constexpr int kAdmmSmemRows = 192;
constexpr unsigned kAdmmSmemBytes = kAdmmSmemRows * kAdmmSmemRows * 4u;
// Dynamic shared memory of the batched contact kernel without ADMM members: W of working sets up to
// 64 rows (two blocks per SM stay resident; larger working sets keep W in global memory).
constexpr unsigned kBatchWSmemBytes = 64u * 64u * 8u;
constexpr int kContactNode = 0, kContactSegment = 1;
// A triangle whose plane projection of the node lies inside it enlarged by this barycentric margin
// ("over the face") gives a constraint row; the same value is used by the CPU oracle.
constexpr double kFaceBand = 0.1;

// Status codes mirrored from accfem.h
enum : int { ST_OK = 0, ST_INVALID = 1, ST_NOMEM = 2, ST_CUDA = 3, ST_NOT_CONVERGED = 4,
             ST_CAPACITY = 5, ST_NOT_SPD = 6, ST_TIMEOUT = 7 };

// Which limit raised ST_CAPACITY (Ctl::cap_code).
enum : int { CAP_ROWS = 1, CAP_CANDIDATES = 2, CAP_SURVIVORS = 3, CAP_NODE_ROWS = 4, CAP_LCP_ROWS = 5,
             CAP_WORKING = 6 };

// Flags of a constraint row, carried from one Newton iteration to the next by (node, triangle):
// active (y > 0), in the working set, violated by the last applied step, violated at some
// iteration of this solve (such a row stays in the working set).
enum : int { RF_ACTIVE = 1, RF_WORKING = 2, RF_VIOLATED = 4, RF_STICKY = 8 };

// Constants of one handle, passed by value to every kernel.
struct Params {
  int M, N;                      // elements, nodes
  double L, l0, EA, EI, GJ, r_o;
  double act, beta0, tol, lcp_tol;
  int max_lcp_iters;
  double e[3];                   // entrance point
  double E0[9];                  // rest triad, row-major, columns = d, up, d x up
  double q0[4];                  // quaternion of E0
  int n_cables;
  double r_c, cable_cos[kMaxCables], cable_sin[kMaxCables];
  // lumen grid (triangles binned by centroid)
  double g_org[3], g_h, g_rq;    // origin, cell size, query half-width
  int g_dim[3];
  int n_tri;
  double eps_d;                  // FP32 distance margin (m)
  float eps_b;                   // FP32 relative barycentric margin
  int m_cap;                     // max constraint rows
  int ws_cap;                    // max rows of the working set (<= kMaxWorking)
  int nrhs_cap;                  // 1 + ws_cap RHS columns
  double ws_gap;                 // a row whose gap is at most this joins the working set
  int ws_all;                    // every constraint row is in the working set (frame mode)
  int max_newton;                // Newton iteration cap of a solve
  int precision;                 // kPrecisionFP64 or kPrecisionMixed (FP32 element tangent)
  int lcp_mode;                  // kLcpActiveSet, or kLcpAdmm (OSQP's ADMM guess, then the exact polish)
  int admm_iters;                // ADMM iteration cap
  int contact_model;             // kContactNode (rows at nodes) or kContactSegment (rows anywhere on an element)
};

// Control block, resident on the device; one per handle.
struct Ctl {
  int k;                 // last prescribed node
  int nf;                // number of free nodes (k+1 .. M)
  int m;                 // constraint rows of the current iteration
  int iter;              // Newton iterations done in this solve
  int converged;
  int status;            // first error (ST_*), 0 if none
  int same_set;          // constraint set identical to the previous iteration
  int m_prev;
  int lcp_pivots;        // LCP pivot steps in this solve
  int n_active;
  int load_mode;         // 0 cables, 1 dead tip load (global), 2 follower tip load (tip frame)
  int loops;             // passes of the device-side Newton loop
  unsigned long long umax_bits, step_bits, res_bits;   // atomicMax on non-negative doubles
  double alpha;          // alpha of the last applied step
  double rho;            // step bound of the limiter (starts at beta0)
  int has_prev;          // a previous Newton step exists in this solve
  int aa_n;              // previous iterates held for the acceleration (0..kAccelDepth)
  int aa_prev;           // the last applied step was an accelerated one
  int n_active_prev;     // active rows of the previous iteration
  int same_active;       // the active rows are those of the previous iteration (by node and triangle)
  double nrm2_prev;      // sum of |du|^2 of the previous step (secant over-relaxation)
  double aa_dmax[kAccelDepth];                  // bound on the largest nodal translation of each held increment
  unsigned long long aa_cmax_bits[kAccelDepth]; // this iteration: largest nodal translation of f_{k-j+1} - f_{k-j}
  // limiter decision of the current iteration, written by the first apply block for the control update
  double lim_rho, lim_alpha, lim_bound, lim_nrm2;
  int lim_accel, lim_steady;
  int live;              // batch: a solve of this instance is in flight
  int cap_code;          // CAP_* cause of an ST_CAPACITY status
  int mc;                // rows of the working set (RHS columns 1..mc)
  int incomplete;        // a row outside the working set is violated by this iteration's step
  int fp64_tangent;      // mixed precision: this solve fell back to the FP64 element tangent
  int admm_iters;        // ADMM iterations of this solve (contact solver kLcpAdmm)
  int frame;             // frame mode: reaching the iteration cap is the normal end of a solve
  double delta;          // insertion of the resident state
  double tension[kMaxCables];
  double tip_f[3], tip_m[3];
};

// Programmatic dependent launch.  A kernel launched with programmatic stream serialization may
// start while its predecessor in the stream is still running: pdl_wait() blocks until that
// predecessor has completed and its writes are visible (a no-op for a kernel launched without the
// attribute), so every such kernel calls it before its first access to global memory.
// pdl_trigger() then lets the successor launch and wait in turn, so that at most one kernel waits
// ahead of the running one.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_enter() { pdl_wait(); pdl_trigger(); }

// Flags ST_CAPACITY (the first error of an iteration wins) and records its cause.
__device__ __forceinline__ void flag_capacity(Ctl* c, int code) {
  if (atomicCAS(&c->status, 0, ST_CAPACITY) == 0) c->cap_code = code;
}

// Device buffers of one handle (all device pointers).
struct Dev {
  double *px, *py, *pz, *qw, *qx, *qy, *qz;          // N nodal poses
  double *ox, *oy, *oz, *ow, *oqx, *oqy, *oqz;       // previous poses (warm start source)
  double* elem;                                      // M * kElemStride
  double* kel;                                       // M * 4: EA/l0, GJ/l0, EI/l0, 0 of element e
  // lumen
  const int* cell_start;                             // ncells + 1
  const float* tri32;                                // T * 9: vertices relative to the cell centre
  const float* sph32;                                // T * 4: bounding sphere (centre rel. cell centre, radius)
  const int* cell_tri;                               // T: triangle id of sorted slot
  const double* V;                                   // n_vertices * 3
  const int* T;                                      // n_tri * 3
  const double* nface;                               // n_tri * 3 outward unit normals
  // per owner constraint lists: owner f = free node f (node rows; node = k + 1 + f) or free element f
  // (segment rows; element k + f, joining nodes k + f and k + 1 + f)
  int* ncon;                                         // nf_cap
  int* con_tri;                                      // nf_cap * kListCap
  double* con_pt;                                    // nf_cap * kListCap * 3 (wall point)
  double* con_n;                                     // nf_cap * kListCap * 3
  double* con_gap;                                   // nf_cap * kListCap
  double* con_s;                                     // nf_cap * kListCap: chord fraction of a segment row
  int* con_keep;                                     // nf_cap: rows of an element kept after the shared-node merge
  // compacted constraint rows.  Row r constrains n^T du(contact point) = w1 . du_{c_node} + w2 . du_{c_node2}
  // (free-node indices; c_node2 = -1: one node): a node row has w1 = n; a segment row of element
  // k + f has c_node = f (the element's far node), c_node2 = f - 1 (-1 when prescribed) and the
  // weights of Eq. 4-6 in the element frame
  int* c_node;                                       // owner f of row (its free node, or the element's far node)
  int* c_tri;
  double *c_pt, *c_n, *c_gap;                        // m_cap * 3, * 3, * 1
  int* c_node2;                                      // m_cap: second node of a segment row, else -1
  double *c_w1, *c_w2;                               // m_cap * 3 each: weights on the two nodes' translations
  double* c_s;                                       // m_cap: chord fraction of a segment row (0 for node rows)
  int *c_first;                                      // nf_cap + 1: rows of node f = [c_first[f], c_first[f+1])
  int *p_node, *p_tri;                               // previous iteration's rows
  int *p_first;                                      // nf_cap + 1: previous rows of node f = [p_first[f], p_first[f+1])
  int *p_flag;                                       // previous rows: RF_* flags
  int *init_flag;                                    // current rows: flags of the same row in the previous iteration, -1 new
  int *wrow;                                         // ws_cap: row of working-set slot k (rows in order)
  int *rslot;                                        // m_cap: working-set slot of row r, -1 outside
  // block-tridiagonal system (free nodes)
  double *D, *U, *P, *Lm, *Rm;                       // nf_cap * 36 each, row-major 6x6
  double* B;                                         // nf_cap * 6 * nrhs_cap, [(f*6+c)*nrhs_cap + r]; column 0 -g,
                                                     // column 1 + k: A^T e_row for working-set slot k
  double* g;                                         // nf_cap * 6 : F - F_a on free DOFs
  double* dx;                                        // nf_cap * 6 : Newton step
  double* du_prev;                                   // nf_cap * 3 : previous Newton step (translations)
  double* rev_part;                                  // per step_kernel block: sum du . du_prev
  double* aa_part;                                   // per step_kernel block: kAccelParts least-squares sums
  double* aa_f;                                      // kAccelSlots * nf_cap * 6: unscaled steps of previous iterates
  double* aa_d;                                      // kAccelSlots * nf_cap * 6: increments applied there
  // contact LCP
  double *W, *y, *gj;                                // ws_cap^2 (slots), m_cap (rows), ws_cap*(ws_cap+2)
  int *plist;                                        // ws_cap: active slots
  // primal ADMM (contact solver kLcpPrimalAdmm, primal.cu): the reduction of K + sigma I + rho A^T A
  double *pa_D, *pa_E, *pa_P, *pa_EL, *pa_ER;        // nf_cap * 36 each
  double *pa_x, *pa_xt, *pa_w, *pa_v;                // nf_cap * 6 each: x, the solve's result, RHS, scratch
  double *pa_z, *pa_lam;                             // m_cap: z and the multipliers of every row
  int* pa_guess;                                     // m_cap: 1 where the multiplier is positive (the guess)
  Ctl* ctl;
};

// ---------------------------------------------------------------- small FP64 helpers
__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]));
}
__device__ __forceinline__ void cross3(const double* a, const double* b, double* c) {
  c[0] = fma(a[1], b[2], -a[2] * b[1]);
  c[1] = fma(a[2], b[0], -a[0] * b[2]);
  c[2] = fma(a[0], b[1], -a[1] * b[0]);
}
__device__ __forceinline__ unsigned long long dbits(double v) {
  return (unsigned long long)__double_as_longlong(v);
}

// Rotation matrix (row-major) of the unit quaternion (w, x, y, z).
__device__ __forceinline__ void quat_to_mat(double w, double x, double y, double z, double* R) {
  double xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y,
         wz = w * z;
  R[0] = 1.0 - 2.0 * (yy + zz); R[1] = 2.0 * (xy - wz);       R[2] = 2.0 * (xz + wy);
  R[3] = 2.0 * (xy + wz);       R[4] = 1.0 - 2.0 * (xx + zz); R[5] = 2.0 * (yz - wx);
  R[6] = 2.0 * (xz - wy);       R[7] = 2.0 * (yz + wx);       R[8] = 1.0 - 2.0 * (xx + yy);
}

// Hamilton product c = a * b.
__device__ __forceinline__ void quat_mul(const double* a, const double* b, double* c) {
  c[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  c[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  c[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  c[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// Rotation vector theta of the rotation matrix R (angle below pi): theta = (t / (2 sin t)) vee(R - R^T).
// The factor t/sin t = asin(s)/s with s = sin t is evaluated by its Taylor series when s^2 < 0.01
// (relative truncation error below 1e-16 with the terms kept), otherwise from atan2.
__device__ __forceinline__ void rotvec_of_mat(const double* R, double* th) {
  double v0 = R[7] - R[5], v1 = R[2] - R[6], v2 = R[3] - R[1];   // 2 sin t * axis
  double s2 = 0.25 * fma(v0, v0, fma(v1, v1, v2 * v2));
  double c = 0.5 * (R[0] + R[4] + R[8] - 1.0);
  double f;
  if (s2 < 1e-2 && c > 0.0) {
    // asin(s)/s = sum_k (2k)! / (4^k (k!)^2 (2k+1)) s^(2k)
    f = fma(s2, 0.01396484375, 0.017352764423076924);     // k=7: 429/30720=0.01396484375, k=6: 231/13312
    f = fma(s2, f, 0.022372159090909092);                 // k=5: 63/2816
    f = fma(s2, f, 0.030381944444444444);                 // k=4: 35/1152
    f = fma(s2, f, 0.044642857142857144);                 // k=3: 5/112
    f = fma(s2, f, 0.075);                                // k=2: 3/40
    f = fma(s2, f, 1.0 / 6.0);                            // k=1
    f = fma(s2, f, 1.0);
    f *= 0.5;
  } else {
    double s = sqrt(s2);
    double t = atan2(s, c);
    f = (s > 0.0) ? 0.5 * t / s : 0.5;
  }
  th[0] = f * v0; th[1] = f * v1; th[2] = f * v2;
}

// Tsinv(theta) = I - [theta]x/2 + eta [theta]x^2, eta = (1 - (t/2) cot(t/2)) / t^2 (row-major 3x3).
// eta by its series 1/12 + t^2/720 + t^4/30240 + t^6/1209600 + t^8/47900160 for t^2 < 0.04.
__device__ __forceinline__ void tsinv_mat(const double* th, double* Ti) {
  double t2 = fma(th[0], th[0], fma(th[1], th[1], th[2] * th[2]));
  double eta;
  if (t2 < 0.04) {
    eta = fma(t2, 1.0 / 47900160.0, 1.0 / 1209600.0);
    eta = fma(t2, eta, 1.0 / 30240.0);
    eta = fma(t2, eta, 1.0 / 720.0);
    eta = fma(t2, eta, 1.0 / 12.0);
  } else {
    double t = sqrt(t2);
    eta = (1.0 - 0.5 * t / tan(0.5 * t)) / t2;
  }
  // [th]x^2 = th th^T - t2 I
  double a = th[0], b = th[1], c = th[2];
  Ti[0] = 1.0 + eta * (a * a - t2); Ti[1] = 0.5 * c + eta * a * b;      Ti[2] = -0.5 * b + eta * a * c;
  Ti[3] = -0.5 * c + eta * a * b;   Ti[4] = 1.0 + eta * (b * b - t2);   Ti[5] = 0.5 * a + eta * b * c;
  Ti[6] = 0.5 * b + eta * a * c;    Ti[7] = -0.5 * a + eta * b * c;     Ti[8] = 1.0 + eta * (c * c - t2);
}

// Unit quaternion of the rotation vector theta: (cos(t/2), sin(t/2)/t theta), series for t^2 < 0.01.
__device__ __forceinline__ void quat_exp(const double* th, double* q) {
  double t2 = fma(th[0], th[0], fma(th[1], th[1], th[2] * th[2]));
  double cw, sf;
  if (t2 < 1e-2) {
    double x = 0.25 * t2;   // (t/2)^2
    // cos(u) = 1 - u^2/2 + u^4/24 - u^6/720 + u^8/40320 - u^10/3628800; sin(u)/u similarly, u = t/2
    cw = fma(x, -1.0 / 3628800.0, 1.0 / 40320.0);
    cw = fma(x, cw, -1.0 / 720.0);
    cw = fma(x, cw, 1.0 / 24.0);
    cw = fma(x, cw, -0.5);
    cw = fma(x, cw, 1.0);
    double su = fma(x, 1.0 / 39916800.0, -1.0 / 362880.0);
    su = fma(x, su, 1.0 / 5040.0);
    su = fma(x, su, -1.0 / 120.0);
    su = fma(x, su, 1.0 / 6.0);
    su = fma(x, -su, 1.0);
    sf = 0.5 * su;            // sin(t/2) / t = (sin(u)/u) / 2
  } else {
    double t = sqrt(t2);
    double s, c;
    sincos(0.5 * t, &s, &c);
    cw = c;
    sf = s / t;
  }
  q[0] = cw; q[1] = sf * th[0]; q[2] = sf * th[1]; q[3] = sf * th[2];
}

// Rotation vector of the unit quaternion q (w >= 0 enforced): 2 asin(|v|)/|v| v, series for |v|^2 < 0.01.
__device__ __forceinline__ void quat_log(const double* qin, double* th) {
  double sg = qin[0] < 0.0 ? -1.0 : 1.0;
  double w = sg * qin[0], x = sg * qin[1], y = sg * qin[2], z = sg * qin[3];
  double s2 = fma(x, x, fma(y, y, z * z));
  double f;
  if (s2 < 1e-2) {
    f = fma(s2, 0.01396484375, 0.017352764423076924);
    f = fma(s2, f, 0.022372159090909092);
    f = fma(s2, f, 0.030381944444444444);
    f = fma(s2, f, 0.044642857142857144);
    f = fma(s2, f, 0.075);
    f = fma(s2, f, 1.0 / 6.0);
    f = fma(s2, f, 1.0);
    f *= 2.0;
  } else {
    double s = sqrt(s2);
    f = 2.0 * atan2(s, w) / s;
  }
  th[0] = f * x; th[1] = f * y; th[2] = f * z;
}

}  // namespace accfem
