// Point-triangle geometry shared by the collision kernels.
#pragma once
#include "common.cuh"

namespace accfem {

// FP32 squared distance from p to triangle (a, b, c) and the unnormalised barycentrics of the
// plane projection (va, vb, vc) with va + vb + vc = |ab x ac|^2.
__device__ __forceinline__ float tri_dist2_f32(const float* p, const float* t, float& va, float& vb, float& vc) {
  float ab[3] = {t[3] - t[0], t[4] - t[1], t[5] - t[2]};
  float ac[3] = {t[6] - t[0], t[7] - t[1], t[8] - t[2]};
  float ap[3] = {p[0] - t[0], p[1] - t[1], p[2] - t[2]};
  float d1 = ab[0] * ap[0] + ab[1] * ap[1] + ab[2] * ap[2];
  float d2 = ac[0] * ap[0] + ac[1] * ap[1] + ac[2] * ap[2];
  float bp[3] = {ap[0] - ab[0], ap[1] - ab[1], ap[2] - ab[2]};
  float d3 = ab[0] * bp[0] + ab[1] * bp[1] + ab[2] * bp[2];
  float d4 = ac[0] * bp[0] + ac[1] * bp[1] + ac[2] * bp[2];
  float cp[3] = {ap[0] - ac[0], ap[1] - ac[1], ap[2] - ac[2]};
  float d5 = ab[0] * cp[0] + ab[1] * cp[1] + ab[2] * cp[2];
  float d6 = ac[0] * cp[0] + ac[1] * cp[1] + ac[2] * cp[2];
  va = d3 * d6 - d5 * d4;
  vb = d5 * d2 - d1 * d6;
  vc = d1 * d4 - d3 * d2;
  float q[3];
  if (d1 <= 0.f && d2 <= 0.f) { q[0] = 0.f; q[1] = 0.f; q[2] = 0.f; }
  else if (d3 >= 0.f && d4 <= d3) { q[0] = ab[0]; q[1] = ab[1]; q[2] = ab[2]; }
  else if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) {
    float v = d1 / (d1 - d3); q[0] = v * ab[0]; q[1] = v * ab[1]; q[2] = v * ab[2];
  } else if (d6 >= 0.f && d5 <= d6) { q[0] = ac[0]; q[1] = ac[1]; q[2] = ac[2]; }
  else if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) {
    float w = d2 / (d2 - d6); q[0] = w * ac[0]; q[1] = w * ac[1]; q[2] = w * ac[2];
  } else if (va <= 0.f && (d4 - d3) >= 0.f && (d5 - d6) >= 0.f) {
    float w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
    q[0] = ab[0] + w * (ac[0] - ab[0]); q[1] = ab[1] + w * (ac[1] - ab[1]); q[2] = ab[2] + w * (ac[2] - ab[2]);
  } else {
    float den = 1.f / (va + vb + vc);
    float v = vb * den, w = vc * den;
    q[0] = v * ab[0] + w * ac[0]; q[1] = v * ab[1] + w * ac[1]; q[2] = v * ab[2] + w * ac[2];
  }
  float r[3] = {ap[0] - q[0], ap[1] - q[1], ap[2] - q[2]};
  return r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
}

// FP64 closest point of triangle (A, B, C) to p (the Voronoi-region method of Ericson, Real-Time
// Collision Detection, 2005, Sec. 5.1.5), with "interior" = all three unnormalised barycentrics of
// the plane projection >= 0 and "near" = all three >= -kFaceBand times their sum.  Returns the
// closest point in c (absolute), |c - p|^2, and the two flags.
static __device__ double tri_closest_f64(const double* p, const double* A, const double* B, const double* C,
                                  double* c, int* interior, int* near) {
  double ab[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
  double ac[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
  double ap[3] = {p[0] - A[0], p[1] - A[1], p[2] - A[2]};
  double bp[3] = {ap[0] - ab[0], ap[1] - ab[1], ap[2] - ab[2]};
  double cp[3] = {ap[0] - ac[0], ap[1] - ac[1], ap[2] - ac[2]};
  double d1 = dot3(ab, ap), d2 = dot3(ac, ap), d3 = dot3(ab, bp), d4 = dot3(ac, bp), d5 = dot3(ab, cp),
         d6 = dot3(ac, cp);
  double va = d3 * d6 - d5 * d4, vb = d5 * d2 - d1 * d6, vc = d1 * d4 - d3 * d2;
  const double band = -kFaceBand * (va + vb + vc);
  *near = (va >= band && vb >= band && vc >= band) ? 1 : 0;
  double q[3];
  *interior = 0;
  if (va >= 0.0 && vb >= 0.0 && vc >= 0.0) {
    *interior = 1;
    double den = __drcp_rn(va + vb + vc);
    double v = vb * den, w = vc * den;
    q[0] = v * ab[0] + w * ac[0]; q[1] = v * ab[1] + w * ac[1]; q[2] = v * ab[2] + w * ac[2];
  } else if (d1 <= 0.0 && d2 <= 0.0) { q[0] = 0.0; q[1] = 0.0; q[2] = 0.0; }
  else if (d3 >= 0.0 && d4 <= d3) { q[0] = ab[0]; q[1] = ab[1]; q[2] = ab[2]; }
  else if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
    double v = d1 / (d1 - d3); q[0] = v * ab[0]; q[1] = v * ab[1]; q[2] = v * ab[2];
  } else if (d6 >= 0.0 && d5 <= d6) { q[0] = ac[0]; q[1] = ac[1]; q[2] = ac[2]; }
  else if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
    double w = d2 / (d2 - d6); q[0] = w * ac[0]; q[1] = w * ac[1]; q[2] = w * ac[2];
  } else {
    double den = (d4 - d3) + (d5 - d6);
    double w = den > 0.0 ? (d4 - d3) / den : 0.0;
    q[0] = ab[0] + w * (ac[0] - ab[0]); q[1] = ab[1] + w * (ac[1] - ab[1]); q[2] = ab[2] + w * (ac[2] - ab[2]);
  }
  double r[3] = {ap[0] - q[0], ap[1] - q[1], ap[2] - q[2]};
  c[0] = A[0] + q[0]; c[1] = A[1] + q[1]; c[2] = A[2] + q[2];
  return dot3(r, r);
}

struct Surv {
  int t;
  int interior;     // plane projection inside the triangle
  int near;         // plane projection inside the triangle enlarged by kFaceBand
  int pad;
  double d2;
  double c[3];
};

}  // namespace accfem
