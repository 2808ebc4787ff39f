// Host-side state of a batch (internal; shared by the batch driver and the request server).
#pragma once
#include <string>
#include <vector>

#include "handle.h"
#include "batch.cuh"

struct accfem_batch {
  std::vector<accfem_handle*> members;
  int n = 0;
  int max_nodes = 0;
  int levels = 0;
  cudaStream_t stream = nullptr, user_stream = nullptr;
  cudaStream_t side = nullptr;      // second branch of an iteration (element phase beside collision)
  cudaEvent_t fork = nullptr, join = nullptr;
  accfem::Inst* d_tab = nullptr;
  accfem::Plan* d_plan = nullptr;
  Ctl* d_ctl = nullptr;             // control block of member i (the batch's own)
  Ctl* d_stage = nullptr;           // staged control blocks of the solves begun since the last advance
  accfem::BatchBegin* d_begin = nullptr;
  int* d_members = nullptr;         // result gather: member list, offsets, packed values
  long long* d_off = nullptr;
  double* d_pack = nullptr;
  size_t pack_cap = 0;              // doubles
  Ctl* h_ctl = nullptr;             // pinned host mirrors
  Ctl* h_stage = nullptr;
  accfem::BatchBegin* h_begin = nullptr;
  int* h_members = nullptr;
  long long* h_off = nullptr;
  double* h_pack = nullptr;
  int* h_passes = nullptr;
  double* d_tips = nullptr;         // request server: tip pose + row count of finished members
  double* h_tips = nullptr;
  int64_t dev_bytes = 0;            // device memory held by the batch itself
  int n_begin = 0;
  std::vector<int> state;           // 0 idle, 1 staged, 2 in flight
  std::vector<int> solved;          // member finished at least one solve in this batch
  // graph variants (built on first use): v % 4 divides the persistent grids by 1, 2, 4 or 8; v / 4
  // picks the element mapping, blocks of 2, 4 or 8 warps with one warp per element
  static constexpr int kVariants = 12;
  int elem_w = 2;                   // warps per element block of the variant being captured or run
  bool has_segment = false;         // a member uses segment contacts (their collision kernel is launched too)
  bool has_admm = false;            // a member uses the ADMM contact solver (contact kernel with its shared memory)
  struct Variant {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int grid[accfem::kPhases] = {};
  };
  Variant variants[kVariants];
  int variant = 0;                  // variant in use
  int tune_left = 0;                // advances left in the autotuning round
  int tune_next = 0;
  double tune_ms[kVariants] = {};
  int64_t tune_passes[kVariants] = {};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int body_kernels = 0;
  bool stream_mode = false;         // ACCFEM_LAUNCH=stream: host-driven passes (kernels visible to profilers)
  bool pdl = false;                 // programmatic dependent launch of the phase kernels (ACCFEM_PDL=1)
  int grid[accfem::kPhases] = {};
  int64_t launches = 0, h2d = 0, d2h = 0;
  std::string err;
  cudaStream_t work() const { return user_stream ? user_stream : stream; }
};

inline accfem_status bfail(accfem_batch* b, accfem_status s, const std::string& msg) {
  if (b) b->err = msg;
  return s;
}

inline bool bok(accfem_batch* b, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return true;
  if (b) b->err = std::string(what) + ": " + cudaGetErrorString(e);
  return false;
}

// Outcome of a finished solve from its control block.
inline accfem_status outcome(const Ctl& c) {
  if (c.status != 0) return (accfem_status)c.status;
  if (c.nf == 0 || c.converged || c.frame) return ACCFEM_OK;
  return ACCFEM_E_NOT_CONVERGED;
}
