// Request server over a batch (accfem_batch_serve, include/accfem.h): continuous batching of timed
// requests.  Each request is one quasi-static solve of a resident scene (batch member), warm
// started from that scene's resident state; requests of one scene run in arrival order, requests of
// different scenes overlap on the device.  The loop admits the requests that have arrived into idle
// scenes, advances everything in flight by a few Newton iterations (one batch graph launch), and
// answers the solves that finished with their tip pose, gathered in one kernel and one copy (and, when
// the caller asks for them, their full results through the batch's result gather).
#include <chrono>
#include <deque>
#include <thread>
#include <vector>

#include "batch_host.h"

namespace accfem {

// Tip pose (x, y, z, qw, qx, qy, qz) and constraint-row count of members[0..count).
__global__ void batch_tip_kernel(const Inst* __restrict__ tab, const int* __restrict__ members, int count, double* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= count) return;
  const Inst& in = tab[members[j]];
  const int t = in.p.M;
  const Ctl* c = in.d.ctl;
  double* o = out + 8 * (size_t)j;
  o[0] = in.d.px[t]; o[1] = in.d.py[t]; o[2] = in.d.pz[t];
  o[3] = in.d.qw[t]; o[4] = in.d.qx[t]; o[5] = in.d.qy[t]; o[6] = in.d.qz[t];
  o[7] = (c->nf > 0 && c->iter > 0) ? (double)c->m : 0.0;
}

}  // namespace accfem

using namespace accfem;

extern "C" {

accfem_status accfem_batch_serve(accfem_batch* b, const accfem_request* requests, int32_t n_requests, int32_t chunk_iters,
                                 int64_t hbm_cap_bytes, accfem_response* responses, accfem_result* results) {
  if (!b) return ACCFEM_E_INVALID_ARG;
  b->err.clear();
  if (n_requests < 0 || chunk_iters < 1 || (n_requests > 0 && (!requests || !responses)))
    return bfail(b, ACCFEM_E_INVALID_ARG, "bad arguments");
  for (int i = 0; i < b->n; ++i)
    if (b->state[i] != 0) return bfail(b, ACCFEM_E_INVALID_ARG, "a member has a solve staged or in flight");
  for (int k = 0; k < n_requests; ++k) {
    const accfem_request& r = requests[k];
    if (r.member < 0 || r.member >= b->n || !(r.arrival >= 0.0) || (k > 0 && r.arrival < requests[k - 1].arrival))
      return bfail(b, ACCFEM_E_INVALID_ARG, "requests need members in range and non-decreasing arrival times");
  }
  // admission by device footprint: the batch itself, then members in index order while they fit
  std::vector<char> admitted(b->n, 0);
  int64_t used = b->dev_bytes;
  for (int i = 0; i < b->n; ++i) {
    const int64_t need = b->members[i]->dev_bytes;
    if (hbm_cap_bytes <= 0 || used + need <= hbm_cap_bytes) {
      admitted[i] = 1;
      used += need;
    }
  }
  std::vector<std::deque<int>> queue(b->n);
  std::vector<int> current(b->n, -1);
  std::vector<int> fin;
  const auto t0 = std::chrono::steady_clock::now();
  auto now = [&]() { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); };
  int next = 0, answered = 0;
  cudaStream_t st = b->work();
  while (answered < n_requests) {
    const double t = now();
    for (; next < n_requests && requests[next].arrival <= t; ++next) {
      const accfem_request& r = requests[next];
      accfem_response& o = responses[next];
      o = accfem_response{};
      if (!admitted[r.member]) {
        o.status = ACCFEM_E_NOMEM;
        o.t_begin = o.t_end = t;
        ++answered;
      } else {
        queue[r.member].push_back(next);
      }
    }
    int flying = 0;
    for (int i = 0; i < b->n; ++i) {
      if (current[i] < 0 && !queue[i].empty()) {
        const int k = queue[i].front();
        queue[i].pop_front();
        const accfem_status s = accfem_batch_begin(b, i, requests[k].cable_tensions, requests[k].insertion);
        responses[k].t_begin = now();
        if (s != ACCFEM_OK) {
          responses[k].status = s;
          responses[k].t_end = responses[k].t_begin;
          ++answered;
          continue;
        }
        current[i] = k;
      }
      flying += current[i] >= 0;
    }
    if (flying == 0) {
      if (next >= n_requests) break;
      while (now() < requests[next].arrival) std::this_thread::yield();
      continue;
    }
    int32_t left = 0;
    accfem_status s = accfem_batch_advance(b, chunk_iters, &left);
    if (s != ACCFEM_OK) return s;
    fin.clear();
    for (int i = 0; i < b->n; ++i)
      if (current[i] >= 0 && b->state[i] == 0) fin.push_back(i);
    if (fin.empty()) continue;
    const int nf = (int)fin.size();
    for (int j = 0; j < nf; ++j) b->h_members[j] = fin[j];
    if (!bok(b, cudaMemcpyAsync(b->d_members, b->h_members, sizeof(int) * nf, cudaMemcpyHostToDevice, st), "upload list"))
      return ACCFEM_E_CUDA;
    batch_tip_kernel<<<(nf + 127) / 128, 128, 0, st>>>(b->d_tab, b->d_members, nf, b->d_tips);
    ++b->launches;
    if (!bok(b, cudaGetLastError(), "gather tips") ||
        !bok(b, cudaMemcpyAsync(b->h_tips, b->d_tips, sizeof(double) * 8 * nf, cudaMemcpyDeviceToHost, st), "download tips") ||
        !bok(b, cudaStreamSynchronize(st), "download tips"))
      return ACCFEM_E_CUDA;
    b->h2d += sizeof(int) * nf;
    b->d2h += sizeof(double) * 8 * nf;
    if (results) {
      // full answers (poses, rows, forces) of the finished solves, into the callers' result buffers
      std::vector<accfem_result> full(nf);
      std::vector<accfem_status> fst(nf);
      for (int j = 0; j < nf; ++j) full[j] = results[current[fin[j]]];
      const accfem_status r = accfem_batch_results(b, fin.data(), nf, full.data(), fst.data());
      if (r == ACCFEM_E_CUDA || r == ACCFEM_E_INVALID_ARG) return r;
      b->err.clear();
      for (int j = 0; j < nf; ++j) results[current[fin[j]]] = full[j];
    }
    const double te = now();
    for (int j = 0; j < nf; ++j) {
      const int i = fin[j], k = current[i];
      accfem_response& o = responses[k];
      const Ctl& c = b->h_ctl[i];
      o.status = outcome(c);
      o.newton_iters = c.iter;
      o.t_end = te;
      for (int a = 0; a < 7; ++a) o.tip[a] = b->h_tips[8 * j + a];
      o.n_contacts = (int32_t)b->h_tips[8 * j + 7];
      current[i] = -1;
      ++answered;
    }
  }
  return ACCFEM_OK;
}

}  // extern "C"
