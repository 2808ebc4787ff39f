// C ABI of the Acc-FEM hot path (see include/accfem.h): handle set-up, lumen grid, and the Newton
// driver that launches the per-iteration kernels on the handle's stream.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>
#include <map>

#include "../../include/accfem.h"
#include "handle.h"
#include "batch.cuh"

namespace accfem {
__global__ void element_kernel(Params p, Dev d);
__global__ void collide_kernel(Params p, Dev d);
__global__ void collide_segment_kernel(Params p, Dev d);
__global__ void compact_kernel(Params p, Dev d);
__global__ void bcr_bwd_kernel(Params p, Dev d, int s, int nf);
__global__ void contact_kernel(Params p, Dev d);
__global__ void step_kernel(Params p, Dev d);
__global__ void apply_kernel(Params p, Dev d);
__global__ void start_kernel(Params p, Dev d, int mode, double delta, double delta_old, int k);
__global__ void ctl_kernel(Params p, Dev d, cudaGraphConditionalHandle h, int max_iter, int set_cond);
__global__ void assemble_rhs_kernel(Params p, Dev d);
__global__ void bcr_level_kernel(Params p, Dev d, int s, int nf);
__global__ void primal_admm_kernel(Params p, Dev d);
void upload_element_tables();
}  // namespace accfem

using namespace accfem;

namespace {

accfem_status fail(accfem_handle* h, accfem_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}

bool cuda_ok(accfem_handle* h, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  if (h) h->err = std::string(what) + ": " + cudaGetErrorString(e);
  return false;
}

template <typename T>
bool dalloc(accfem_handle* h, T** ptr, size_t count) {
  void* p = nullptr;
  if (count == 0) count = 1;
  if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
    h->err = "cudaMalloc failed";
    return false;
  }
  cudaMemset(p, 0, count * sizeof(T));
  h->allocs.push_back(p);
  h->dev_bytes += (int64_t)(count * sizeof(T));
  *ptr = (T*)p;
  return true;
}

void quat_of_matrix(const double* R, double* q) {   // R row-major, Shepperd branch choice, w >= 0
  double tr = R[0] + R[4] + R[8];
  double c[4] = {tr, R[0], R[4], R[8]};
  int k = 0;
  for (int i = 1; i < 4; ++i)
    if (c[i] > c[k]) k = i;
  if (k == 0) {
    double w = 0.5 * std::sqrt(1.0 + tr);
    q[0] = w; q[1] = (R[7] - R[5]) / (4 * w); q[2] = (R[2] - R[6]) / (4 * w); q[3] = (R[3] - R[1]) / (4 * w);
  } else if (k == 1) {
    double x = 0.5 * std::sqrt(1.0 + 2 * R[0] - tr);
    q[0] = (R[7] - R[5]) / (4 * x); q[1] = x; q[2] = (R[1] + R[3]) / (4 * x); q[3] = (R[2] + R[6]) / (4 * x);
  } else if (k == 2) {
    double y = 0.5 * std::sqrt(1.0 + 2 * R[4] - tr);
    q[0] = (R[2] - R[6]) / (4 * y); q[1] = (R[1] + R[3]) / (4 * y); q[2] = y; q[3] = (R[5] + R[7]) / (4 * y);
  } else {
    double z = 0.5 * std::sqrt(1.0 + 2 * R[8] - tr);
    q[0] = (R[3] - R[1]) / (4 * z); q[1] = (R[2] + R[6]) / (4 * z); q[2] = (R[5] + R[7]) / (4 * z); q[3] = z;
  }
  if (q[0] < 0) for (int i = 0; i < 4; ++i) q[i] = -q[i];
  double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int i = 0; i < 4; ++i) q[i] /= n;
}

}  // namespace

extern "C" {

const char* accfem_status_string(accfem_status s) {
  switch (s) {
    case ACCFEM_OK: return "ok";
    case ACCFEM_E_INVALID_ARG: return "invalid argument";
    case ACCFEM_E_NOMEM: return "out of memory";
    case ACCFEM_E_CUDA: return "CUDA error";
    case ACCFEM_E_NOT_CONVERGED: return "Newton iterations did not converge";
    case ACCFEM_E_CONTACT_CAPACITY: return "contact capacity exceeded";
    case ACCFEM_E_NOT_SPD: return "tangent or contact matrix not positive definite";
    case ACCFEM_E_TIMEOUT: return "contact LCP pivot limit reached";
    case ACCFEM_E_PENETRATION: return "penetration at convergence";
  }
  return "unknown status";
}

const char* accfem_last_error(const accfem_handle* h) { return h ? h->err.c_str() : ""; }

int64_t accfem_kernel_launches(const accfem_handle* h) { return h ? h->launches : 0; }

accfem_status accfem_default_options(accfem_options* o) {
  if (!o) return ACCFEM_E_INVALID_ARG;
  o->activation_gap = 1.0e-3;
  o->step_limit = 5.0e-4;
  o->newton_tol = 1.0e-11;
  o->contact_tol = 1.0e-11;
  o->max_newton_iters = 200;
  o->max_contact_iters = 1000;
  o->max_contacts = 256;
  o->tangent_mode = 0;
  return ACCFEM_OK;
}

void accfem_destroy(accfem_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& kv : h->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  for (void* p : h->allocs) cudaFree(p);
  if (h->h_ctl) cudaFreeHost(h->h_ctl);
  if (h->h_stage) cudaFreeHost(h->h_stage);
  if (h->fork) cudaEventDestroy(h->fork);
  if (h->join) cudaEventDestroy(h->join);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

accfem_status accfem_create(const accfem_robot_desc* robot, const accfem_lumen_desc* lumen,
                            const accfem_options* options, accfem_handle** out) {
  if (!out) return ACCFEM_E_INVALID_ARG;
  *out = nullptr;
  if (!robot || !lumen) return ACCFEM_E_INVALID_ARG;
  accfem_options opt;
  accfem_default_options(&opt);
  if (options) opt = *options;
  const auto& r = *robot;
  if (!(r.length > 0) || !(r.outer_radius > 0) || !(r.inner_radius >= 0) || !(r.inner_radius < r.outer_radius) ||
      !(r.youngs_modulus > 0) || !(r.poisson_ratio > -1.0 && r.poisson_ratio < 0.5) || r.n_elements < 1 ||
      r.n_elements > (1 << 20) || r.n_cables < 0 || r.n_cables > kMaxCables || (r.n_cables > 0 && !r.cable_angles) ||
      !(r.cable_radius >= 0))
    return ACCFEM_E_INVALID_ARG;
  if (lumen->n_vertices < 0 || lumen->n_triangles < 0 || lumen->n_triangles > (int64_t)INT32_MAX / 3 ||
      (lumen->n_triangles > 0 && (!lumen->vertices || !lumen->triangles)))
    return ACCFEM_E_INVALID_ARG;
  if (!(opt.activation_gap >= 0) || !(opt.step_limit > 0) || !(opt.newton_tol > 0) || !(opt.contact_tol >= 0) ||
      opt.max_newton_iters < 1 || opt.max_contact_iters < 1 || opt.max_contacts < 1 || opt.max_contacts > 8192 ||
      opt.tangent_mode != 0)
    return ACCFEM_E_INVALID_ARG;
  // entrance frame
  double dvec[3] = {lumen->entrance_dir[0], lumen->entrance_dir[1], lumen->entrance_dir[2]};
  double dn = std::sqrt(dvec[0] * dvec[0] + dvec[1] * dvec[1] + dvec[2] * dvec[2]);
  if (!(dn > 0)) return ACCFEM_E_INVALID_ARG;
  for (double& v : dvec) v /= dn;
  double up[3] = {lumen->entrance_up[0], lumen->entrance_up[1], lumen->entrance_up[2]};
  double ud = up[0] * dvec[0] + up[1] * dvec[1] + up[2] * dvec[2];
  for (int i = 0; i < 3; ++i) up[i] -= ud * dvec[i];
  double un = std::sqrt(up[0] * up[0] + up[1] * up[1] + up[2] * up[2]);
  if (!(un > 1e-12)) return ACCFEM_E_INVALID_ARG;
  for (double& v : up) v /= un;
  double th[3] = {dvec[1] * up[2] - dvec[2] * up[1], dvec[2] * up[0] - dvec[0] * up[2], dvec[0] * up[1] - dvec[1] * up[0]};

  accfem_handle* h = new accfem_handle();
  Params& p = h->p;
  std::memset(&p, 0, sizeof(p));
  p.M = r.n_elements;
  p.N = r.n_elements + 1;
  p.L = r.length;
  p.l0 = r.length / r.n_elements;
  const double PI = 3.14159265358979323846;
  double A = PI * (r.outer_radius * r.outer_radius - r.inner_radius * r.inner_radius);
  double I = PI * (std::pow(r.outer_radius, 4) - std::pow(r.inner_radius, 4)) / 4.0;
  double G = r.youngs_modulus / (2.0 * (1.0 + r.poisson_ratio));
  p.EA = r.youngs_modulus * A;
  p.EI = r.youngs_modulus * I;
  p.GJ = G * 2.0 * I;
  h->youngs = r.youngs_modulus;
  h->poisson = r.poisson_ratio;
  h->area = A;
  h->inertia = I;
  p.r_o = r.outer_radius;
  p.act = opt.activation_gap;
  p.beta0 = opt.step_limit;
  p.tol = opt.newton_tol;
  p.lcp_tol = opt.contact_tol;
  p.max_lcp_iters = opt.max_contact_iters;
  for (int i = 0; i < 3; ++i) p.e[i] = lumen->entrance_point[i];
  for (int i = 0; i < 3; ++i) { p.E0[3 * i] = dvec[i]; p.E0[3 * i + 1] = up[i]; p.E0[3 * i + 2] = th[i]; }
  quat_of_matrix(p.E0, p.q0);
  p.n_cables = r.n_cables;
  p.r_c = r.cable_radius;
  for (int j = 0; j < r.n_cables; ++j) { p.cable_cos[j] = std::cos(r.cable_angles[j]); p.cable_sin[j] = std::sin(r.cable_angles[j]); }
  p.m_cap = opt.max_contacts;
  p.ws_cap = std::min(opt.max_contacts, kMaxWorking);
  p.nrhs_cap = p.ws_cap + 1;
  p.ws_gap = 0.2 * opt.step_limit;
  p.eps_d = 1e-6;
  p.eps_b = 1e-3f;
  p.max_newton = opt.max_newton_iters;
  p.lcp_mode = kLcpActiveSet;
  p.admm_iters = 4000;
  h->nf_cap = p.M;
  h->max_newton = opt.max_newton_iters;
  h->max_newton_opt = opt.max_newton_iters;
  {
    const char* lm = std::getenv("ACCFEM_LAUNCH");
    h->stream_mode = lm && std::strcmp(lm, "stream") == 0;
    h->pdl = pdl_default();
    const char* tr = std::getenv("ACCFEM_TRACE");
    h->trace = tr && tr[0] == '1';
  }

  // ---- lumen grid (host): triangles binned by centroid
  const int64_t T = lumen->n_triangles;
  const int64_t NV = lumen->n_vertices;
  std::vector<double> cen(3 * T), nface(3 * T);
  double rmax = 0.0;
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
  for (int64_t t = 0; t < T; ++t) {
    const int32_t* tv = lumen->triangles + 3 * t;
    for (int k = 0; k < 3; ++k)
      if (tv[k] < 0 || tv[k] >= NV) { delete h; return ACCFEM_E_INVALID_ARG; }
    const double* a = lumen->vertices + 3 * tv[0];
    const double* b = lumen->vertices + 3 * tv[1];
    const double* c = lumen->vertices + 3 * tv[2];
    double ab[3], ac[3], n[3];
    for (int k = 0; k < 3; ++k) { ab[k] = b[k] - a[k]; ac[k] = c[k] - a[k]; cen[3 * t + k] = (a[k] + b[k] + c[k]) / 3.0; }
    n[0] = ab[1] * ac[2] - ab[2] * ac[1]; n[1] = ab[2] * ac[0] - ab[0] * ac[2]; n[2] = ab[0] * ac[1] - ab[1] * ac[0];
    double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (!(nn > 0) || !std::isfinite(nn)) { delete h; return ACCFEM_E_INVALID_ARG; }
    for (int k = 0; k < 3; ++k) nface[3 * t + k] = n[k] / nn;
    for (const double* v : {a, b, c}) {
      double dx = v[0] - cen[3 * t], dy = v[1] - cen[3 * t + 1], dz = v[2] - cen[3 * t + 2];
      rmax = std::max(rmax, std::sqrt(dx * dx + dy * dy + dz * dz));
    }
    for (int k = 0; k < 3; ++k) {
      if (t == 0 || cen[3 * t + k] < lo[k]) lo[k] = cen[3 * t + k];
      if (t == 0 || cen[3 * t + k] > hi[k]) hi[k] = cen[3 * t + k];
    }
  }
  p.g_rq = p.r_o + p.act + rmax + 1e-9;
  double hcell = p.g_rq;
  int64_t ncell = 1;
  for (int it = 0; it < 64; ++it) {
    ncell = 1;
    for (int k = 0; k < 3; ++k) {
      p.g_dim[k] = (int)std::floor((hi[k] - lo[k]) / hcell) + 1;
      ncell *= p.g_dim[k];
    }
    if (ncell <= (int64_t)(1 << 24)) break;
    hcell *= 1.26;
  }
  p.g_h = hcell;
  for (int k = 0; k < 3; ++k) p.g_org[k] = lo[k];
  p.n_tri = (int)T;
  std::vector<int> cell_of(T), cstart(ncell + 1, 0), ctri(T);
  for (int64_t t = 0; t < T; ++t) {
    int ci[3];
    for (int k = 0; k < 3; ++k) {
      ci[k] = (int)std::floor((cen[3 * t + k] - p.g_org[k]) / p.g_h);
      ci[k] = std::min(std::max(ci[k], 0), p.g_dim[k] - 1);
    }
    cell_of[t] = (ci[2] * p.g_dim[1] + ci[1]) * p.g_dim[0] + ci[0];
    cstart[cell_of[t] + 1]++;
  }
  for (int64_t c = 0; c < ncell; ++c) cstart[c + 1] += cstart[c];
  {
    std::vector<int> fillp(cstart.begin(), cstart.end() - 1);
    for (int64_t t = 0; t < T; ++t) ctri[fillp[cell_of[t]]++] = (int)t;
  }
  std::vector<float> tri32(9 * std::max<int64_t>(T, 1));
  std::vector<float> sph32(4 * std::max<int64_t>(T, 1));
  for (int64_t c = 0; c < ncell; ++c) {
    int cz = (int)(c / ((int64_t)p.g_dim[0] * p.g_dim[1]));
    int cy = (int)((c / p.g_dim[0]) % p.g_dim[1]);
    int cx = (int)(c % p.g_dim[0]);
    double ctr[3] = {p.g_org[0] + (cx + 0.5) * p.g_h, p.g_org[1] + (cy + 0.5) * p.g_h, p.g_org[2] + (cz + 0.5) * p.g_h};
    for (int s = cstart[c]; s < cstart[c + 1]; ++s) {
      const int64_t t = ctri[s];
      const int32_t* tv = lumen->triangles + 3 * t;
      for (int v = 0; v < 3; ++v)
        for (int k = 0; k < 3; ++k) tri32[9 * (int64_t)s + 3 * v + k] = (float)(lumen->vertices[3 * tv[v] + k] - ctr[k]);
      // bounding sphere about the centroid, radius rounded up so the FP32 test stays conservative
      double rad = 0.0;
      for (int v = 0; v < 3; ++v) {
        double dx = lumen->vertices[3 * tv[v]] - cen[3 * t], dy = lumen->vertices[3 * tv[v] + 1] - cen[3 * t + 1],
               dz = lumen->vertices[3 * tv[v] + 2] - cen[3 * t + 2];
        rad = std::max(rad, std::sqrt(dx * dx + dy * dy + dz * dz));
      }
      for (int k = 0; k < 3; ++k) sph32[4 * (int64_t)s + k] = (float)(cen[3 * t + k] - ctr[k]);
      sph32[4 * (int64_t)s + 3] = (float)(rad * (1.0 + 1e-6) + 1e-9);
    }
  }

  // ---- device memory
  if (!cuda_ok(h, cudaGetDevice(&h->device), "cudaGetDevice") ||
      !cuda_ok(h, cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking), "cudaStreamCreate") ||
      !cuda_ok(h, cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking), "cudaStreamCreate") ||
      !cuda_ok(h, cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming), "cudaEventCreate") ||
      !cuda_ok(h, cudaEventCreateWithFlags(&h->join, cudaEventDisableTiming), "cudaEventCreate")) {
    accfem_destroy(h);
    return ACCFEM_E_CUDA;
  }
  // dynamic shared memory of the contact kernel (beside the LCP's static arrays): W of the active-set
  // LCP, or the contact-space ADMM's FP32 inverse
  if (!cuda_ok(h, cudaFuncSetAttribute(contact_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kAdmmSmemBytes),
               "contact kernel shared memory")) {
    accfem_destroy(h);
    return ACCFEM_E_CUDA;
  }
  upload_element_tables();
  Dev& d = h->d;
  const int N = p.N, M = p.M, nfc = h->nf_cap, mc = p.m_cap, wc = p.ws_cap;
  bool ok = dalloc(h, &d.px, N) && dalloc(h, &d.py, N) && dalloc(h, &d.pz, N) && dalloc(h, &d.qw, N) &&
            dalloc(h, &d.qx, N) && dalloc(h, &d.qy, N) && dalloc(h, &d.qz, N) && dalloc(h, &d.ox, N) &&
            dalloc(h, &d.oy, N) && dalloc(h, &d.oz, N) && dalloc(h, &d.ow, N) && dalloc(h, &d.oqx, N) &&
            dalloc(h, &d.oqy, N) && dalloc(h, &d.oqz, N) && dalloc(h, &d.elem, (size_t)M * kElemStride) &&
            dalloc(h, &d.kel, (size_t)M * 4);
  int *cs = nullptr, *ct = nullptr, *tv = nullptr;
  float* t32 = nullptr;
  float* s32 = nullptr;
  double *vv = nullptr, *nfc_d = nullptr;
  ok = ok && dalloc(h, &cs, ncell + 1) && dalloc(h, &ct, std::max<int64_t>(T, 1)) && dalloc(h, &t32, tri32.size()) && dalloc(h, &s32, sph32.size()) &&
       dalloc(h, &vv, std::max<int64_t>(3 * NV, 1)) && dalloc(h, &tv, std::max<int64_t>(3 * T, 1)) &&
       dalloc(h, &nfc_d, std::max<int64_t>(3 * T, 1));
  ok = ok && dalloc(h, &d.ncon, nfc) && dalloc(h, &d.con_tri, (size_t)nfc * kListCap) &&
       dalloc(h, &d.con_pt, (size_t)nfc * kListCap * 3) && dalloc(h, &d.con_n, (size_t)nfc * kListCap * 3) &&
       dalloc(h, &d.con_gap, (size_t)nfc * kListCap) && dalloc(h, &d.c_node, mc) && dalloc(h, &d.c_tri, mc) &&
       dalloc(h, &d.con_s, (size_t)nfc * kListCap) && dalloc(h, &d.con_keep, nfc) && dalloc(h, &d.c_node2, mc) && dalloc(h, &d.c_w1, (size_t)mc * 3) &&
       dalloc(h, &d.c_w2, (size_t)mc * 3) && dalloc(h, &d.c_s, mc) &&
       dalloc(h, &d.c_pt, 3 * mc) && dalloc(h, &d.c_n, 3 * mc) && dalloc(h, &d.c_gap, mc) &&
       dalloc(h, &d.c_first, nfc + 1) && dalloc(h, &d.p_node, mc) && dalloc(h, &d.p_tri, mc) && dalloc(h, &d.p_first, nfc + 1) &&
       dalloc(h, &d.p_flag, mc) && dalloc(h, &d.init_flag, mc) && dalloc(h, &d.wrow, wc) &&
       dalloc(h, &d.rslot, mc) &&
       dalloc(h, &d.D, (size_t)nfc * 36) && dalloc(h, &d.U, (size_t)nfc * 36) && dalloc(h, &d.P, (size_t)nfc * 36) &&
       dalloc(h, &d.Lm, (size_t)nfc * 36) && dalloc(h, &d.Rm, (size_t)nfc * 36) &&
       dalloc(h, &d.B, (size_t)nfc * 6 * p.nrhs_cap) && dalloc(h, &d.g, (size_t)nfc * 6) &&
       dalloc(h, &d.dx, (size_t)nfc * 6) && dalloc(h, &d.du_prev, (size_t)nfc * 3) &&
       dalloc(h, &d.rev_part, (size_t)nfc / 32 + 2) && dalloc(h, &d.aa_part, ((size_t)nfc / 32 + 2) * kAccelParts) &&
       dalloc(h, &d.aa_f, (size_t)kAccelSlots * nfc * 6) && dalloc(h, &d.aa_d, (size_t)kAccelSlots * nfc * 6) && dalloc(h, &d.W, (size_t)wc * wc) &&
       dalloc(h, &d.y, mc) && dalloc(h, &d.gj, (size_t)wc * (wc + 2)) && dalloc(h, &d.plist, wc) &&
       dalloc(h, &d.pa_D, (size_t)nfc * 36) && dalloc(h, &d.pa_E, (size_t)nfc * 36) && dalloc(h, &d.pa_P, (size_t)nfc * 36) &&
       dalloc(h, &d.pa_EL, (size_t)nfc * 36) && dalloc(h, &d.pa_ER, (size_t)nfc * 36) && dalloc(h, &d.pa_x, (size_t)nfc * 6) &&
       dalloc(h, &d.pa_xt, (size_t)nfc * 6) && dalloc(h, &d.pa_w, (size_t)nfc * 6) && dalloc(h, &d.pa_v, (size_t)nfc * 6) &&
       dalloc(h, &d.pa_z, mc) && dalloc(h, &d.pa_lam, mc) && dalloc(h, &d.pa_guess, mc) &&
       dalloc(h, &d.ctl, 1);
  if (!ok) {
    accfem_destroy(h);
    return ACCFEM_E_NOMEM;
  }
  ok = cuda_ok(h, cudaMemcpy(cs, cstart.data(), sizeof(int) * (ncell + 1), cudaMemcpyHostToDevice), "upload grid") &&
       (T == 0 || cuda_ok(h, cudaMemcpy(ct, ctri.data(), sizeof(int) * T, cudaMemcpyHostToDevice), "upload grid")) &&
       (T == 0 || cuda_ok(h, cudaMemcpy(t32, tri32.data(), sizeof(float) * 9 * T, cudaMemcpyHostToDevice), "upload grid")) &&
       (T == 0 || cuda_ok(h, cudaMemcpy(s32, sph32.data(), sizeof(float) * 4 * T, cudaMemcpyHostToDevice), "upload grid")) &&
       (NV == 0 || cuda_ok(h, cudaMemcpy(vv, lumen->vertices, sizeof(double) * 3 * NV, cudaMemcpyHostToDevice), "upload mesh")) &&
       (T == 0 || cuda_ok(h, cudaMemcpy(tv, lumen->triangles, sizeof(int) * 3 * T, cudaMemcpyHostToDevice), "upload mesh")) &&
       (T == 0 || cuda_ok(h, cudaMemcpy(nfc_d, nface.data(), sizeof(double) * 3 * T, cudaMemcpyHostToDevice), "upload mesh"));
  if (!ok) {
    accfem_destroy(h);
    return ACCFEM_E_CUDA;
  }
  if (accfem_set_element_modulus(h, nullptr, M) != ACCFEM_OK) { accfem_destroy(h); return ACCFEM_E_CUDA; }
  d.cell_start = cs; d.cell_tri = ct; d.tri32 = t32; d.sph32 = s32; d.V = vv; d.T = tv; d.nface = nfc_d;
  if (cudaMallocHost(&h->h_ctl, sizeof(Ctl)) != cudaSuccess) { accfem_destroy(h); return ACCFEM_E_NOMEM; }
  h->stage_bytes = sizeof(double) * (size_t)std::max<int64_t>(7 * N, 16 * (int64_t)mc + 64);
  if (cudaMallocHost(&h->h_stage, h->stage_bytes) != cudaSuccess) { accfem_destroy(h); return ACCFEM_E_NOMEM; }
  std::memset(h->h_ctl, 0, sizeof(Ctl));
  *out = h;
  return ACCFEM_OK;
}

}  // extern "C"

namespace {

#define LAUNCH(h, ...)                                  \
  do {                                                  \
    __VA_ARGS__;                                        \
    ++(h)->launches;                                    \
  } while (0)

// Enqueues the kernels of one Newton iteration for nf free nodes on stream st; returns the count.
// Assembly and RHS columns, then the block cyclic reduction: level-1 eliminations, one kernel per
// level s that updates the kept nodes, eliminates the next level's nodes (or the root) and reduces
// the RHS, and the back substitution.  Returns the number of kernels.
int enqueue_factor(const Params& p, const Dev& d, int nf, cudaStream_t st, bool pdl) {
  int n = 0;
  auto grid = [nf](int ph) { return dim3(phase_gx(ph, nf), phase_gy(ph)); };
  launch_k(pdl, assemble_rhs_kernel, grid(PH_ASM), dim3(32, 6), st, p, d); ++n;
  // the paper's OSQP on the primal QP: its guess of the active rows, before the reduction overwrites D
  if (p.lcp_mode == kLcpPrimalAdmm) { launch_k(pdl, primal_admm_kernel, dim3(1), dim3(1024), st, p, d); ++n; }
  int levels = 0;
  while (levels < kMaxLevels && phase_gx(PH_LEV0 + levels, nf) > 0) ++levels;
  for (int j = 0; j < levels; ++j) { launch_k(pdl, bcr_level_kernel, grid(PH_LEV0 + j), dim3(192), st, p, d, 1 << j, nf); ++n; }
  for (int j = levels - 1; j >= 0; --j)
    if (phase_gx(PH_BWD0 + j, nf) > 0) { launch_k(pdl, bcr_bwd_kernel, grid(PH_BWD0 + j), dim3(96), st, p, d, 1 << j, nf); ++n; }
  return n;
}

int enqueue_iteration(accfem_handle* h, int nf, cudaStream_t st, cudaGraphConditionalHandle cond) {
  Params& p = h->p;
  Dev& d = h->d;
  int n = 0;
  auto grid = [nf](int ph) { return dim3(phase_gx(ph, nf), phase_gy(ph)); };
  // the element kernel and the collision + compaction both only read the poses: two branches that
  // join before the assembly (captured as parallel graph nodes)
  cudaEventRecord(h->fork, st);
  cudaStreamWaitEvent(h->side, h->fork, 0);
  const bool pdl = h->pdl;
  launch_k(pdl, element_kernel, grid(PH_ELEM), dim3(32 * kWarpsPerElemBlock), h->side, p, d); ++n;
  cudaEventRecord(h->join, h->side);
  if (p.contact_model == kContactSegment) launch_k(pdl, collide_segment_kernel, dim3(nf), dim3(128), st, p, d);
  else launch_k(pdl, collide_kernel, grid(PH_COLL), dim3(128), st, p, d);
  ++n;
  launch_k(pdl, compact_kernel, dim3(1), dim3(1024), st, p, d); ++n;
  cudaStreamWaitEvent(st, h->join, 0);
  n += enqueue_factor(p, d, nf, st, pdl);
  launch_ks(pdl, contact_kernel, dim3(1), dim3(256), kAdmmSmemBytes, st, p, d); ++n;
  launch_k(pdl, step_kernel, grid(PH_STEP), dim3(32, 6), st, p, d); ++n;
  launch_k(pdl, apply_kernel, grid(PH_APPLY), dim3(128), st, p, d); ++n;
  launch_k(pdl, ctl_kernel, dim3(1), dim3(1), st, p, d, cond, h->max_newton, h->stream_mode ? 0 : 1); ++n;
  return n;
}

// Device-side Newton loop for nf free nodes: a graph whose WHILE node runs the iteration body until
// ctl_kernel clears the condition (converged, error, or the iteration cap).  Built once per nf.
const accfem_handle::LoopGraph* newton_graph(accfem_handle* h, int nf) {
  auto it = h->graphs.find(nf);
  if (it != h->graphs.end()) return &it->second;
  accfem_handle::LoopGraph lg;
  cudaGraphConditionalHandle cond;
  cudaGraphNodeParams cp = {};
  cudaGraphNode_t node;
  if (!cuda_ok(h, cudaGraphCreate(&lg.graph, 0), "cudaGraphCreate") ||
      !cuda_ok(h, cudaGraphConditionalHandleCreate(&cond, lg.graph, 1, cudaGraphCondAssignDefault), "conditional handle"))
    return nullptr;
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  if (!cuda_ok(h, cudaGraphAddNode(&node, lg.graph, nullptr, nullptr, 0, &cp), "conditional node")) {
    cudaGraphDestroy(lg.graph);
    return nullptr;
  }
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  if (!cuda_ok(h, cudaStreamBeginCaptureToGraph(h->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed),
               "begin capture")) {
    cudaGraphDestroy(lg.graph);
    return nullptr;
  }
  lg.body_kernels = enqueue_iteration(h, nf, h->stream, cond);
  cudaError_t ce = cudaStreamEndCapture(h->stream, &body);
  if (!cuda_ok(h, ce, "end capture") || !cuda_ok(h, cudaGraphInstantiate(&lg.exec, lg.graph, 0), "instantiate graph")) {
    cudaGetLastError();
    cudaGraphDestroy(lg.graph);
    if (h->pdl) {                 // programmatic edges refused inside the loop body: capture without them
      std::fprintf(stderr, "accfem: programmatic dependent launch refused in the Newton graph; plain launches\n");
      h->pdl = false;
      return newton_graph(h, nf);
    }
    return nullptr;
  }
  auto res = h->graphs.emplace(nf, lg);
  return &res.first->second;
}

// Runs one solve on the device; the solution stays resident.  Returns the status.
accfem_status run_solve(accfem_handle* h, int load_mode, const double* tensions_host, const double* tensions_dev,
                        const double* tip_f, const double* tip_m, double insertion, const accfem_state* warm) {
  Params& p = h->p;
  Dev& d = h->d;
  if (!accfem_on_device(h, "solve")) return ACCFEM_E_INVALID_ARG;
  if (!(insertion >= 0.0 && insertion <= p.L)) return fail(h, ACCFEM_E_INVALID_ARG, "insertion outside [0, length]");
  const int k = std::min(std::max(accfem_last_prescribed(p.L, p.M, insertion), 0), p.M);
  const int nf = p.M - k;
  Ctl& c = *h->h_ctl;
  std::memset(&c, 0, sizeof(Ctl));
  c.k = k;
  c.nf = nf;
  c.m_prev = -1;
  c.rho = p.beta0;
  c.load_mode = load_mode;
  c.delta = insertion;
  c.frame = h->frame_iters > 0 ? 1 : 0;
  if (load_mode == 0 && tensions_host) {
    for (int j = 0; j < p.n_cables; ++j) {
      if (!(tensions_host[j] >= 0.0) || !std::isfinite(tensions_host[j]))
        return fail(h, ACCFEM_E_INVALID_ARG, "cable tensions must be finite and non-negative");
      c.tension[j] = tensions_host[j];
    }
  }
  if (load_mode != 0)
    for (int a = 0; a < 3; ++a) {
      if (!std::isfinite(tip_f[a]) || !std::isfinite(tip_m[a])) return fail(h, ACCFEM_E_INVALID_ARG, "tip load not finite");
      c.tip_f[a] = tip_f[a];
      c.tip_m[a] = tip_m[a];
    }
  cudaStream_t st = h->work();
  if (!cuda_ok(h, cudaMemcpyAsync(d.ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, st), "upload control")) return ACCFEM_E_CUDA;
  h->h2d += sizeof(Ctl);
  if (load_mode == 0 && tensions_dev && p.n_cables > 0) {
    if (!cuda_ok(h, cudaMemcpyAsync(&d.ctl->tension[0], tensions_dev, sizeof(double) * p.n_cables, cudaMemcpyDeviceToDevice, st),
                 "copy tensions"))
      return ACCFEM_E_CUDA;
  }
  int mode = 0;
  const size_t nb = sizeof(double) * p.N;
  if (warm) {
    if (!warm->node_pos || !warm->node_quat) return fail(h, ACCFEM_E_INVALID_ARG, "warm state has NULL arrays");
    double* s = h->h_stage;
    for (int comp = 0; comp < 7; ++comp)
      for (int i = 0; i < p.N; ++i)
        s[comp * p.N + i] = comp < 3 ? warm->node_pos[3 * i + comp] : warm->node_quat[4 * i + comp - 3];
    double* dst[7] = {d.px, d.py, d.pz, d.qw, d.qx, d.qy, d.qz};
    for (int comp = 0; comp < 7; ++comp)
      if (!cuda_ok(h, cudaMemcpyAsync(dst[comp], s + comp * p.N, nb, cudaMemcpyHostToDevice, st), "upload warm state"))
        return ACCFEM_E_CUDA;
    h->h2d += 7 * nb;
    mode = 2;
  } else if (h->has_state) {
    double* src[7] = {d.px, d.py, d.pz, d.qw, d.qx, d.qy, d.qz};
    double* dst[7] = {d.ox, d.oy, d.oz, d.ow, d.oqx, d.oqy, d.oqz};
    for (int comp = 0; comp < 7; ++comp)
      if (!cuda_ok(h, cudaMemcpyAsync(dst[comp], src[comp], nb, cudaMemcpyDeviceToDevice, st), "copy state")) return ACCFEM_E_CUDA;
    mode = 1;
  }
  LAUNCH(h, start_kernel<<<(p.N + 127) / 128, 128, 0, st>>>(p, d, mode, insertion, h->delta, k));
  h->has_state = true;
  h->delta = insertion;
  accfem_status status = ACCFEM_OK;
  if (nf > 0 && h->stream_mode) {
    status = ACCFEM_E_NOT_CONVERGED;
    for (int it = 0; it < h->max_newton; ++it) {
      h->launches += enqueue_iteration(h, nf, st, cudaGraphConditionalHandle());
      if (!cuda_ok(h, cudaGetLastError(), "kernel launch") ||
          !cuda_ok(h, cudaMemcpyAsync(h->h_ctl, d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st), "read control") ||
          !cuda_ok(h, cudaStreamSynchronize(st), "Newton iteration"))
        return ACCFEM_E_CUDA;
      h->d2h += sizeof(Ctl);
      if (h->trace)
        std::fprintf(stderr, "accfem it %d alpha %.4f umax %.3e step %.3e res %.3e m %d working %d same %d "
                     "incomplete %d active %d lcp %d\n",
                     c.iter, c.alpha, __builtin_bit_cast(double, (unsigned long long)c.umax_bits),
                     __builtin_bit_cast(double, (unsigned long long)c.step_bits),
                     __builtin_bit_cast(double, (unsigned long long)c.res_bits), c.m, c.mc, c.same_set, c.incomplete,
                     c.n_active, c.lcp_pivots);
      if (c.status != 0) {
        status = (accfem_status)c.status;
        h->err = accfem_solve_message(c, status);
        break;
      }
      if (c.converged) { status = ACCFEM_OK; break; }
    }
    if (status == ACCFEM_E_NOT_CONVERGED && c.frame) status = ACCFEM_OK;
  } else if (nf > 0) {
    const accfem_handle::LoopGraph* lg = newton_graph(h, nf);
    if (!lg) return ACCFEM_E_CUDA;
    if (!cuda_ok(h, cudaGraphLaunch(lg->exec, st), "launch Newton graph") ||
        !cuda_ok(h, cudaMemcpyAsync(h->h_ctl, d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st), "read control") ||
        !cuda_ok(h, cudaStreamSynchronize(st), "Newton loop"))
      return ACCFEM_E_CUDA;
    h->d2h += sizeof(Ctl);
    h->launches += (int64_t)c.loops * lg->body_kernels;
    if (c.status != 0) status = (accfem_status)c.status;
    else if (c.converged || c.frame) status = ACCFEM_OK;
    else status = ACCFEM_E_NOT_CONVERGED;
    if (status != ACCFEM_OK) h->err = accfem_solve_message(c, status);
  } else {
    if (!cuda_ok(h, cudaMemcpyAsync(h->h_ctl, d.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st), "read control") ||
        !cuda_ok(h, cudaStreamSynchronize(st), "start pose"))
      return ACCFEM_E_CUDA;
    h->d2h += sizeof(Ctl);
  }
  return status;
}

// Copies the resident solution into *out.
accfem_status download(accfem_handle* h, accfem_status status, accfem_result* out) {
  Params& p = h->p;
  Dev& d = h->d;
  Ctl& c = *h->h_ctl;
  cudaStream_t st = h->work();
  const int N = p.N;
  double* s = h->h_stage;
  h->d2h += 7 * sizeof(double) * (size_t)N;
  const double* src[7] = {d.px, d.py, d.pz, d.qw, d.qx, d.qy, d.qz};
  for (int comp = 0; comp < 7; ++comp)
    if (!cuda_ok(h, cudaMemcpyAsync(s + comp * N, src[comp], sizeof(double) * N, cudaMemcpyDeviceToHost, st), "download state"))
      return ACCFEM_E_CUDA;
  if (!cuda_ok(h, cudaStreamSynchronize(st), "download state")) return ACCFEM_E_CUDA;
  if (out->node_pos)
    for (int i = 0; i < N; ++i)
      for (int a = 0; a < 3; ++a) out->node_pos[3 * i + a] = s[a * N + i];
  if (out->node_quat)
    for (int i = 0; i < N; ++i)
      for (int a = 0; a < 4; ++a) out->node_quat[4 * i + a] = s[(3 + a) * N + i];
  out->newton_iters = c.iter;
  out->contact_iters = c.lcp_pivots;
  out->residual = c.nf > 0 ? __builtin_bit_cast(double, (unsigned long long)c.res_bits) : 0.0;
  for (int a = 0; a < 6; ++a) out->base_reaction[a] = 0.0;
  const int m = (c.nf > 0 && c.iter > 0) ? c.m : 0;
  out->n_contacts = m;
  if (c.nf > 0 && c.iter > 0) {
    // base reaction: F(x) at the last prescribed node = element k's a-end force/moment
    if (!cuda_ok(h, cudaMemcpyAsync(s, d.elem + (size_t)c.k * kElemStride + 78, sizeof(double) * 6, cudaMemcpyDeviceToHost, st),
                 "download reaction"))
      return ACCFEM_E_CUDA;
    if (!cuda_ok(h, cudaStreamSynchronize(st), "download reaction")) return ACCFEM_E_CUDA;
    for (int a = 0; a < 6; ++a) out->base_reaction[a] = s[a];
    h->d2h += 6 * sizeof(double);
  }
  if (m > 0) {
    const int nw = std::min(m, std::max(out->contact_capacity, 0));
    if (nw > 0) {
      std::vector<int> node(m), tri(m);
      std::vector<double> pt(3 * m), nn(3 * m), y(m);
      bool ok = cuda_ok(h, cudaMemcpyAsync(node.data(), d.c_node, sizeof(int) * m, cudaMemcpyDeviceToHost, st), "download") &&
                cuda_ok(h, cudaMemcpyAsync(tri.data(), d.c_tri, sizeof(int) * m, cudaMemcpyDeviceToHost, st), "download") &&
                cuda_ok(h, cudaMemcpyAsync(pt.data(), d.c_pt, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost, st), "download") &&
                cuda_ok(h, cudaMemcpyAsync(nn.data(), d.c_n, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost, st), "download") &&
                cuda_ok(h, cudaMemcpyAsync(y.data(), d.y, sizeof(double) * m, cudaMemcpyDeviceToHost, st), "download") &&
                cuda_ok(h, cudaStreamSynchronize(st), "download contacts");
      if (!ok) return ACCFEM_E_CUDA;
      h->d2h += (size_t)m * (2 * sizeof(int) + 7 * sizeof(double));
      for (int i = 0; i < nw; ++i) {
        if (out->contact_node) out->contact_node[i] = c.k + 1 + node[i];
        if (out->contact_tri) out->contact_tri[i] = tri[i];
        for (int a = 0; a < 3; ++a) {
          if (out->contact_point) out->contact_point[3 * i + a] = pt[3 * i + a];
          if (out->contact_normal) out->contact_normal[3 * i + a] = nn[3 * i + a];
        }
        if (out->contact_force) out->contact_force[i] = y[i];
      }
    }
    if (m > out->contact_capacity && status == ACCFEM_OK) {
      h->err = "result contact capacity too small";
      return ACCFEM_E_CONTACT_CAPACITY;
    }
  }
  return status;
}

}  // namespace

extern "C" {

accfem_status accfem_solve(accfem_handle* h, const double* cable_tensions, double insertion, const accfem_state* warm,
                           accfem_result* out) {
  if (!h || !out || (h->p.n_cables > 0 && !cable_tensions)) return fail(h, ACCFEM_E_INVALID_ARG, "NULL argument");
  h->err.clear();
  accfem_status s = run_solve(h, 0, cable_tensions, nullptr, nullptr, nullptr, insertion, warm);
  if (s == ACCFEM_E_INVALID_ARG || s == ACCFEM_E_CUDA) return s;
  return download(h, s, out);
}

accfem_status accfem_solve_tip_load(accfem_handle* h, const double f[3], const double m[3], int32_t follower,
                                    double insertion, const accfem_state* warm, accfem_result* out) {
  if (!h || !out || !f || !m) return fail(h, ACCFEM_E_INVALID_ARG, "NULL argument");
  h->err.clear();
  accfem_status s = run_solve(h, follower ? 2 : 1, nullptr, nullptr, f, m, insertion, warm);
  if (s == ACCFEM_E_INVALID_ARG || s == ACCFEM_E_CUDA) return s;
  return download(h, s, out);
}

accfem_status accfem_solve_resident(accfem_handle* h, const double* device_cable_tensions, double insertion,
                                    int32_t* newton_iters) {
  if (!h || (h->p.n_cables > 0 && !device_cable_tensions)) return fail(h, ACCFEM_E_INVALID_ARG, "NULL argument");
  h->err.clear();
  accfem_status s = run_solve(h, 0, nullptr, device_cable_tensions, nullptr, nullptr, insertion, nullptr);
  if (newton_iters) *newton_iters = h->h_ctl->iter;
  return s;
}

accfem_status accfem_reset(accfem_handle* h) {
  if (!h) return ACCFEM_E_INVALID_ARG;
  h->has_state = false;
  h->delta = 0.0;
  return ACCFEM_OK;
}

accfem_status accfem_set_precision(accfem_handle* h, int32_t mode) {
  if (!h || (mode != ACCFEM_PRECISION_FP64 && mode != ACCFEM_PRECISION_MIXED)) return ACCFEM_E_INVALID_ARG;
  if (h->p.precision == mode) return ACCFEM_OK;
  if (h->stream) cudaStreamSynchronize(h->work());
  for (auto& kv : h->graphs) {     // the Newton graphs captured the handle's constants
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  h->graphs.clear();
  h->p.precision = mode;
  return ACCFEM_OK;
}

accfem_status accfem_set_contact_solver(accfem_handle* h, int32_t solver) {
  if (!h || (solver != ACCFEM_CONTACT_ACTIVE_SET && solver != ACCFEM_CONTACT_ADMM && solver != ACCFEM_CONTACT_PRIMAL_ADMM))
    return ACCFEM_E_INVALID_ARG;
  if (solver == ACCFEM_CONTACT_PRIMAL_ADMM && h->p.contact_model != kContactNode)
    return fail(h, ACCFEM_E_INVALID_ARG, "the primal ADMM takes node contacts only");
  if (h->p.lcp_mode == solver) return ACCFEM_OK;
  if (h->stream) cudaStreamSynchronize(h->work());
  for (auto& kv : h->graphs) {     // the Newton graphs captured the handle's constants
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  h->graphs.clear();
  h->p.lcp_mode = solver == ACCFEM_CONTACT_ADMM ? kLcpAdmm : solver == ACCFEM_CONTACT_PRIMAL_ADMM ? kLcpPrimalAdmm : kLcpActiveSet;
  return ACCFEM_OK;
}

accfem_status accfem_set_contact_model(accfem_handle* h, int32_t model) {
  if (!h || (model != ACCFEM_CONTACT_NODE && model != ACCFEM_CONTACT_SEGMENT)) return ACCFEM_E_INVALID_ARG;
  if (model == ACCFEM_CONTACT_SEGMENT && h->p.lcp_mode == kLcpPrimalAdmm)
    return fail(h, ACCFEM_E_INVALID_ARG, "the primal ADMM takes node contacts only");
  if (h->p.contact_model == model) return ACCFEM_OK;
  if (h->stream) cudaStreamSynchronize(h->work());
  for (auto& kv : h->graphs) {     // the Newton graphs captured the collision kernel of the model
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  h->graphs.clear();
  h->p.contact_model = model == ACCFEM_CONTACT_SEGMENT ? kContactSegment : kContactNode;
  return ACCFEM_OK;
}

accfem_status accfem_set_frame_mode(accfem_handle* h, int32_t iters_per_frame) {
  if (!h || iters_per_frame < 0 || iters_per_frame > 1000000) return ACCFEM_E_INVALID_ARG;
  if (h->frame_iters == iters_per_frame) return ACCFEM_OK;
  if (h->stream) cudaStreamSynchronize(h->work());
  for (auto& kv : h->graphs) {     // the Newton graphs captured the iteration cap and the constants
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  h->graphs.clear();
  h->frame_iters = iters_per_frame;
  h->max_newton = iters_per_frame > 0 ? iters_per_frame : h->max_newton_opt;
  h->p.max_newton = h->max_newton;
  h->p.ws_all = iters_per_frame > 0 ? 1 : 0;
  return ACCFEM_OK;
}

accfem_status accfem_set_element_modulus(accfem_handle* h, const double* youngs_modulus, int32_t n_elements) {
  if (!h || n_elements != h->p.M) return ACCFEM_E_INVALID_ARG;
  const int M = h->p.M;
  std::vector<double> k(4 * (size_t)M, 0.0);
  for (int e = 0; e < M; ++e) {
    const double E = youngs_modulus ? youngs_modulus[e] : h->youngs;
    if (!(E > 0.0) || !std::isfinite(E)) return ACCFEM_E_INVALID_ARG;
    // section constants of Sec. II.B with this element's modulus; E = the robot's gives p.EA etc.
    const double EA = youngs_modulus ? E * h->area : h->p.EA;
    const double EI = youngs_modulus ? E * h->inertia : h->p.EI;
    const double GJ = youngs_modulus ? E / (2.0 * (1.0 + h->poisson)) * 2.0 * h->inertia : h->p.GJ;
    k[4 * e] = EA / h->p.l0;
    k[4 * e + 1] = GJ / h->p.l0;
    k[4 * e + 2] = EI / h->p.l0;
  }
  if (h->stream) cudaStreamSynchronize(h->work());
  if (!cuda_ok(h, cudaMemcpy(h->d.kel, k.data(), sizeof(double) * k.size(), cudaMemcpyHostToDevice), "upload moduli"))
    return ACCFEM_E_CUDA;
  h->h2d += (int64_t)(sizeof(double) * k.size());
  return ACCFEM_OK;
}

accfem_status accfem_set_stream(accfem_handle* h, void* stream) {
  if (!h) return ACCFEM_E_INVALID_ARG;
  h->user_stream = (cudaStream_t)stream;
  return ACCFEM_OK;
}

accfem_status accfem_transfer_bytes(const accfem_handle* h, int64_t* h2d, int64_t* d2h) {
  if (!h || !h2d || !d2h) return ACCFEM_E_INVALID_ARG;
  *h2d = h->h2d;
  *d2h = h->d2h;
  return ACCFEM_OK;
}

}  // extern "C"

namespace {

// accfem_time_kernel (graph = false: reps host launches of the kernel or sequence) and
// accfem_time_kernel_graph (graph = true: reps copies captured in sequence into one CUDA graph,
// replayed once untimed and once timed).
accfem_status time_kernel(accfem_handle* h, accfem_kernel kernel, int32_t reps, double* us, bool graph) {
  const char* who = graph ? "accfem_time_kernel_graph" : "accfem_time_kernel";
  if (!h || !us || reps < 1) return fail(h, ACCFEM_E_INVALID_ARG, "NULL argument or reps < 1");
  if (!accfem_on_device(h, who)) return ACCFEM_E_INVALID_ARG;
  Params& p = h->p;
  Dev& d = h->d;
  Ctl& c = *h->h_ctl;
  const int nf = c.nf;
  if (nf <= 0 || !h->has_state) return fail(h, ACCFEM_E_INVALID_ARG, "no resident solve with free nodes");
  if ((kernel == ACCFEM_KERNEL_CONTACT || kernel == ACCFEM_KERNEL_FACTOR) && c.iter < 1)
    return fail(h, ACCFEM_E_INVALID_ARG, "no completed iteration");
  if (kernel < ACCFEM_KERNEL_ELEMENT || kernel > ACCFEM_KERNEL_FACTOR) return fail(h, ACCFEM_E_INVALID_ARG, "unknown kernel");
  cudaStream_t st = h->work();
  // the kernels return early on a converged control block: run them on a copy flagged "iterating"
  Ctl run = c;
  run.converged = 0;
  run.status = 0;
  if (!cuda_ok(h, cudaMemcpyAsync(d.ctl, &run, sizeof(Ctl), cudaMemcpyHostToDevice, st), "upload control")) return ACCFEM_E_CUDA;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int per_launch = 1;
  auto launch = [&]() {
    switch (kernel) {
      case ACCFEM_KERNEL_ELEMENT:
        element_kernel<<<phase_gx(PH_ELEM, nf), 32 * kWarpsPerElemBlock, 0, st>>>(p, d); break;
      case ACCFEM_KERNEL_COLLIDE:
        if (p.contact_model == kContactSegment) collide_segment_kernel<<<nf, 128, 0, st>>>(p, d);
        else collide_kernel<<<phase_gx(PH_COLL, nf), 128, 0, st>>>(p, d);
        break;
      case ACCFEM_KERNEL_ASSEMBLE:
        assemble_rhs_kernel<<<dim3(phase_gx(PH_ASM, nf), phase_gy(PH_ASM)), dim3(32, 6), 0, st>>>(p, d); break;
      case ACCFEM_KERNEL_FACTOR: per_launch = enqueue_factor(p, d, nf, st, h->pdl); break;
      default: contact_kernel<<<1, 256, kAdmmSmemBytes, st>>>(p, d); break;
    }
  };
  launch();
  bool ok = true;
  if (!graph) {
    cudaEventRecord(e0, st);
    for (int i = 0; i < reps; ++i) launch();
    cudaEventRecord(e1, st);
    h->launches += (int64_t)(reps + 1) * per_launch;
  } else {
    // the capture records the launches without running them; the graph then runs twice
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    ok = cuda_ok(h, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (ok) {
      for (int i = 0; i < reps; ++i) launch();
      ok = cuda_ok(h, cudaStreamEndCapture(st, &g), "end capture") &&
           cuda_ok(h, cudaGraphInstantiate(&ge, g, 0), "instantiate graph") &&
           cuda_ok(h, cudaGraphLaunch(ge, st), "graph launch");
      if (ok) {
        cudaEventRecord(e0, st);
        ok = cuda_ok(h, cudaGraphLaunch(ge, st), "graph launch");
        cudaEventRecord(e1, st);
      }
    }
    h->launches += (int64_t)(2 * reps + 1) * per_launch;
    if (ge) cudaGraphExecDestroy(ge);
    if (g) cudaGraphDestroy(g);
  }
  ok = ok && cuda_ok(h, cudaEventSynchronize(e1), "time kernel");
  float ms = 0.f;
  if (ok) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // restore the control block of the solve (also after a failed capture)
  const bool restored = cuda_ok(h, cudaMemcpyAsync(d.ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, st), "restore control") &&
                        cuda_ok(h, cudaStreamSynchronize(st), "restore control");
  if (!ok || !restored) return ACCFEM_E_CUDA;
  *us = 1000.0 * ms / reps;
  return ACCFEM_OK;
}

}  // namespace

extern "C" {

accfem_status accfem_time_kernel(accfem_handle* h, accfem_kernel kernel, int32_t reps, double* us) {
  return time_kernel(h, kernel, reps, us, false);
}

accfem_status accfem_time_kernel_graph(accfem_handle* h, accfem_kernel kernel, int32_t reps, double* us) {
  return time_kernel(h, kernel, reps, us, true);
}

accfem_status accfem_solve_stats(const accfem_handle* h, int32_t* rows, int32_t* working_rows, int32_t* active_rows,
                                 int32_t* fp64_fallback) {
  if (!h) return ACCFEM_E_INVALID_ARG;
  const Ctl& c = *h->h_ctl;
  const bool it = c.nf > 0 && c.iter > 0;
  if (rows) *rows = it ? c.m : 0;
  if (working_rows) *working_rows = it ? c.mc : 0;
  if (active_rows) *active_rows = it ? c.n_active : 0;
  if (fp64_fallback) *fp64_fallback = c.fp64_tangent;
  return ACCFEM_OK;
}

accfem_status accfem_solve_admm_iterations(const accfem_handle* h, int32_t* iters) {
  if (!h || !iters) return ACCFEM_E_INVALID_ARG;
  *iters = h->h_ctl->admm_iters;
  return ACCFEM_OK;
}

accfem_status accfem_device_bytes(const accfem_handle* h, int64_t* bytes) {
  if (!h || !bytes) return ACCFEM_E_INVALID_ARG;
  *bytes = h->dev_bytes;
  return ACCFEM_OK;
}

accfem_status accfem_get_state(accfem_handle* h, double* node_pos, double* node_quat) {
  if (!h || !node_pos || !node_quat) return fail(h, ACCFEM_E_INVALID_ARG, "NULL argument");
  if (!accfem_on_device(h, "accfem_get_state")) return ACCFEM_E_INVALID_ARG;
  accfem_result r;
  std::memset(&r, 0, sizeof(r));
  r.node_pos = node_pos;
  r.node_quat = node_quat;
  Ctl saved = *h->h_ctl;
  h->h_ctl->nf = 0;   // poses only
  accfem_status s = download(h, ACCFEM_OK, &r);
  *h->h_ctl = saved;
  return s;
}

}  // extern "C"

// Internal views used by the allocation-free collision query (noalloc.cu).
bool accfem_internal_views(accfem_handle* h, Params* p, Dev* d, cudaStream_t* stream) {
  if (!h) return false;
  *p = h->p;
  *d = h->d;
  *stream = h->work();
  return true;
}

void accfem_internal_set_error(accfem_handle* h, const char* msg) {
  if (h) h->err = msg ? msg : "";
}

bool accfem_internal_on_device(accfem_handle* h, const char* who) { return h && accfem_on_device(h, who); }
