// Replica exchange (parallel tempering) over the replica batch: G groups of M
// chains, each group holding one chain at each temperature of a geometric
// ladder T_0 < ... < T_{M-1}.  The paper runs many chains of its sampler in
// parallel (Sections III-C, IV-A) without saying how they interact; replica
// exchange is one standard way to let them: between blocks of sweeps, the
// chains at neighbouring temperatures of a group may trade temperatures.
//
// Exchange round e tries the pairs (m, m+1) with m = e mod 2, m+2, ... of
// every group.  With a the chain at level m and b the one at m+1, the trade
// is accepted with probability min(1, exp((1/T_m - 1/T_{m+1})(E_a - E_b))),
// i.e. iff X = E_b - E_a <= 0, or X < len_m and u < thr_m[X], where thr_m is
// the Metropolis table at the pair's effective temperature
// T_m T_{m+1} / (T_{m+1} - T_m) and u is word 0 of Philox4x32-10 at counter
// (m, e, g, 0x50545843) under the run's key.  The pairs of one round are
// disjoint, so one thread decides each.  Chains keep their states; a trade
// swaps the chains' level entries and the ladder's owner entries.
#include "qp_device.cuh"
#include "qp_internal.h"

namespace qp {
namespace {

constexpr uint32_t kPtTag = 0x50545843u;

__global__ void k_pt_exchange(PtArgs a) {
  const int R = a.G * a.M;
  const int P = (a.M - a.phase) / 2;  // pairs per group this round
  const int pairs = a.G * P;
  const int total = R > pairs ? R : pairs;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += gridDim.x * blockDim.x) {
    if (idx < R && a.best_seg) {
      const int64_t b = a.best_seg[idx];
      if (b < a.best[idx]) a.best[idx] = b;
    }
    if (idx < pairs) {
      const int g = idx / P, m = a.phase + 2 * (idx % P);
      const int ia = g * a.M + m;
      const int ra = a.owner[ia], rb = a.owner[ia + 1];
      const int64_t X = a.E[rb] - a.E[ra];
      bool take = X <= 0;
      if (!take && X < (int64_t)a.len[m]) {
        const uint4 u = dev::philox4x32_10(make_uint4((uint32_t)m, (uint32_t)a.round, (uint32_t)g, kPtTag),
                                           a.key0, a.key1);
        take = u.x < a.thr[a.off[m] + X];
      }
      if (take) {
        a.owner[ia] = rb;
        a.owner[ia + 1] = ra;
        a.level[ra] = m + 1;
        a.level[rb] = m;
        a.swaps[(size_t)g * (a.M - 1) + m] += 1;
      }
    }
  }
}

}  // namespace

cudaError_t launch_pt_exchange(const PtArgs &a, cudaStream_t st) {
  const int R = a.G * a.M;
  const int threads = 256;
  const int blocks = (R + threads - 1) / threads;
  k_pt_exchange<<<blocks < 1 ? 1 : blocks, threads, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace qp
