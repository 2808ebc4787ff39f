// Host-side state of one handle (internal; shared by the single-instance driver and the batch).
#pragma once
#include <cmath>
#include <cstdlib>
#include <map>
#include <string>
#include <vector>

#include "../../include/accfem.h"
#include "common.cuh"

using accfem::Params;
using accfem::Dev;
using accfem::Ctl;

struct accfem_handle {
  Params p;
  Dev d;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;       // second branch of an iteration (element kernel beside collision)
  cudaEvent_t fork = nullptr, join = nullptr;
  std::vector<void*> allocs;
  Ctl* h_ctl = nullptr;            // pinned host mirror of the control block
  double* h_stage = nullptr;       // pinned staging for results
  size_t stage_bytes = 0;
  bool has_state = false;
  double delta = 0.0;
  int64_t launches = 0;
  int nf_cap = 0;
  int max_newton = 200;              // iteration cap of a solve (the frame's in frame mode)
  int max_newton_opt = 200;          // the options' cap
  int frame_iters = 0;               // frame mode: Newton iterations per solve, 0 = solve to convergence
  std::string err;
  struct LoopGraph { cudaGraph_t graph = nullptr; cudaGraphExec_t exec = nullptr; int body_kernels = 0; };
  std::map<int, LoopGraph> graphs;   // device-side Newton loop, one per number of free nodes
  bool stream_mode = false;          // ACCFEM_LAUNCH=stream: host-driven loop (kernels visible to profilers)
  bool pdl = false;                  // programmatic dependent launch of the iteration kernels (ACCFEM_PDL=1)
  bool trace = false;                // ACCFEM_TRACE=1 (with stream mode): one line per Newton iteration on stderr
  cudaStream_t user_stream = nullptr; // caller's stream (accfem_set_stream), else the handle's own
  int64_t h2d = 0, d2h = 0;          // bytes copied by solve / state calls
  int64_t dev_bytes = 0;             // device memory held by the handle
  int device = -1;                   // CUDA device the handle was created on (all its memory lives there)
  double youngs = 0.0, poisson = 0.0, area = 0.0, inertia = 0.0;   // robot material and section
  cudaStream_t work() const { return user_stream ? user_stream : stream; }
};

// Launches kernel<<<grid, block, smem, st>>>(args...); with pdl, as a programmatic dependent launch
// (the kernel may start while its predecessor in st finishes; every kernel of the Newton iteration
// waits for its predecessor in its first instruction, pdl_wait).
template <typename... K, typename... A>
inline void launch_ks(bool pdl, void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = pdl ? attr : nullptr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <typename... K, typename... A>
inline void launch_k(bool pdl, void (*kernel)(K...), dim3 grid, dim3 block, cudaStream_t st, A... args) {
  launch_ks(pdl, kernel, grid, block, 0, st, args...);
}

// Programmatic dependent launch of the iteration kernels: off unless ACCFEM_PDL=1.  Measured on the
// 600 mm, 300-element insertion sweep: with host-issued launches it cuts the factor group by about
// 30% at 10-80 free nodes, but inside the conditional-graph Newton loop the sweep runs 13% slower
// than with the graph's own kernel-to-kernel dependencies.
inline bool pdl_default() {
  const char* v = std::getenv("ACCFEM_PDL");
  return v && v[0] == '1';
}

// True when the current CUDA device is the one the handle was created on; otherwise records a message
// naming `who` and returns false (kernels launched on another device would read this handle's
// pointers as foreign addresses).
inline bool accfem_on_device(accfem_handle* h, const char* who) {
  int dev = -1;
  if (cudaGetDevice(&dev) == cudaSuccess && dev == h->device) return true;
  h->err = std::string(who) + ": the current CUDA device (" + std::to_string(dev) +
           ") is not the device the handle was created on (" + std::to_string(h->device) + ")";
  return false;
}

// Last prescribed node at insertion delta: nodes 0..k sit in the feeder, k = floor((L - delta) M / L).
inline int accfem_last_prescribed(double L, int M, double delta) {
  return (int)std::floor((L - delta) * M / L + 1e-6);
}

// Message of a solve's failure status, with the limit that raised a capacity error.
inline std::string accfem_solve_message(const Ctl& c, accfem_status s) {
  std::string m = accfem_status_string(s);
  if (s == ACCFEM_E_CONTACT_CAPACITY) {
    switch (c.cap_code) {
      case accfem::CAP_ROWS: m += ": constraint rows above max_contacts"; break;
      case accfem::CAP_CANDIDATES: m += ": a node has more than 768 triangles within the activation distance"; break;
      case accfem::CAP_SURVIVORS: m += ": a node has more than 64 triangles for the exact distance test"; break;
      case accfem::CAP_NODE_ROWS: m += ": a node has more than 16 constraint rows (an element more than 32 in the segment model)"; break;
      case accfem::CAP_LCP_ROWS: m += ": working-set rows above the contact solver's 512"; break;
      case accfem::CAP_WORKING: m += ": working-set rows above min(max_contacts, 512)"; break;
      default: break;
    }
  }
  return m;
}
