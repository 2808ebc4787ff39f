// Batched execution of independent instances (handles): one launch per Newton phase advances every
// instance that still iterates.  Each phase kernel is persistent: its blocks walk a packed list of
// work units (instance, block of that instance) built on the device at the end of every iteration
// from the instances still iterating, so converged instances cost nothing.  A unit runs the same
// block body as the single-instance kernel of that phase, so one instance gives identical results
// alone and in a batch.
#pragma once
#include "common.cuh"

namespace accfem {

constexpr int kMaxBatch = 1024;     // instances per batch
constexpr int kMaxLevels = 21;      // reduction strides 1 .. 2^20 (n_elements <= 2^20)

struct Inst {
  Params p;
  Dev d;
};

// Phases of one Newton iteration; level j of the reduction has stride s = 2^j.
enum : int {
  PH_ELEM = 0, PH_COLL, PH_COMPACT, PH_ASM, PH_CONTACT, PH_STEP, PH_APPLY,
  PH_LEV0,
  PH_BWD0 = PH_LEV0 + kMaxLevels,
  kPhases = PH_BWD0 + kMaxLevels
};

// Work plan of the current iteration: the iterating instances and, per phase, the exclusive prefix
// of their unit counts (pre[ph][j] = first unit of the j-th iterating instance).
struct Plan {
  int n_act;
  int passes;                        // iterations run by the current advance
  int max_passes;                    // iteration budget of the current advance
  int act[kMaxBatch];
  int pre[kPhases][kMaxBatch + 1];
};

// A solve that starts in the next advance: start pose mode (0 straight, 1 follow the resident path),
// insertion and the previous insertion, last prescribed node.
struct BatchBegin {
  int member, mode, k, pad;
  double delta, delta_old;
};

// Blocks in x of phase ph for nf free nodes (the single-instance launch uses the same grid).
__host__ __device__ inline int phase_gx(int ph, int nf) {
  if (nf <= 0) return 0;
  switch (ph) {
    case PH_ELEM: return (nf + kWarpsPerElemBlock - 1) / kWarpsPerElemBlock;
    case PH_COLL: return (nf + 3) / 4;
    case PH_COMPACT: return 1;
    case PH_ASM: return nf;
    case PH_CONTACT: return 1;
    case PH_STEP: return (nf + 31) / 32;
    case PH_APPLY: return (nf + 127) / 128;
    default: break;
  }
  if (ph >= PH_LEV0 && ph < PH_BWD0) {
    const int j = ph - PH_LEV0;
    const long long s = 1ll << j;
    if (s < nf) return (int)((nf - 1) / (2 * s) + 1);
    return (j == 0 && nf == 1) ? 1 : 0;       // a single free node: the root step alone
  }
  if (ph >= PH_BWD0 && ph < kPhases) {
    const long long s = 1ll << (ph - PH_BWD0);
    return s < nf ? (int)((nf - s - 1) / (2 * s) + 1) : 0;
  }
  return 0;
}

// Blocks in y (RHS column split) of phase ph; a level launch has one more block in y, which does the
// 6x6 block work of its node while the others reduce the RHS.
__host__ __device__ inline int phase_gy(int ph) {
  if (ph >= PH_LEV0 && ph < PH_BWD0) return kRhsSplit + 1;
  if (ph >= PH_BWD0 && ph < kPhases) return kBwdSplit;
  return ph == PH_ASM ? kRhsSplit : 1;
}

// Persistent loop over the units of phase ph: body(inst, bx, by) for every unit assigned to this
// block (units w = blockIdx.x, blockIdx.x + gridDim.x, ...), with a block barrier between units.
// Every thread of the block runs the same sequence of units.
template <class Body>
__device__ __forceinline__ void for_units(const Inst* __restrict__ tab, const Plan* __restrict__ plan, int ph, Body body) {
  __shared__ int s_pre[kMaxBatch + 1];
  pdl_enter();
  const int na = plan->n_act;
  const int total = plan->pre[ph][na];
  if ((int)blockIdx.x >= total) return;
  for (int i = threadIdx.x + threadIdx.y * blockDim.x; i <= na; i += blockDim.x * blockDim.y) s_pre[i] = plan->pre[ph][i];
  __syncthreads();
  int j = 0;
  for (int w = blockIdx.x; w < total; w += gridDim.x) {
    while (s_pre[j + 1] <= w) ++j;              // units are visited in increasing order
    const int inst = plan->act[j];
    const int l = w - s_pre[j];
    const int gx = phase_gx(ph, tab[inst].d.ctl->nf);
    body(tab[inst], l % gx, l / gx);
    __syncthreads();
  }
}

}  // namespace accfem
