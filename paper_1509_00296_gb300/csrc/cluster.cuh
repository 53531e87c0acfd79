// Split-K reductions across a grid of thread-block clusters (sm_90+).
//
// A cluster first sums its member CTAs' partials through distributed shared
// memory; the cluster that finishes last (atomic ticket, no spin-wait) then sums
// the per-cluster partials in a fixed order, so results are deterministic.
#pragma once
#include <cooperative_groups.h>

#include "common.cuh"

namespace frsvt {

constexpr int kCL = 8;   // CTAs per cluster (portable size)

// part_sm: this CTA's partial (count elements, shared).  cpart: [nclusters][count] global
// scratch.  out: the final sum (count, global).  Returns true in the CTAs of the cluster that
// finished last; they have written `out` (fenced) when the call returns.
template <typename T, int CL = kCL>
__device__ bool cluster_split_reduce(T* part_sm, int count, T* cpart, T* out, unsigned* ticket, int cluster_idx,
                                     int nclusters, int* flag_sm) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = static_cast<int>(cl.block_rank());
  cl.sync();
  const int per = (count + CL - 1) / CL;
  const int e0 = rank * per;
  const int e1 = min(count, e0 + per);
  for (int e = e0 + static_cast<int>(threadIdx.x); e < e1; e += blockDim.x) {
    T v[CL];
#pragma unroll
    for (int r = 0; r < CL; ++r) v[r] = cl.map_shared_rank(part_sm, r)[e];
    T s = 0;
#pragma unroll
    for (int r = 0; r < CL; ++r) s += v[r];
    cpart[static_cast<int64_t>(cluster_idx) * count + e] = s;
  }
  __threadfence();
  cl.sync();
  if (rank == 0 && threadIdx.x == 0) {
    const unsigned old = atomicAdd(ticket, 1u);
    *flag_sm = (old == static_cast<unsigned>(nclusters - 1)) ? 1 : 0;
  }
  cl.sync();
  const int last = *cl.map_shared_rank(flag_sm, 0);
  cl.sync();                                   // rank 0's flag is read before anyone leaves
  if (!last) return false;
  __threadfence();
  for (int e = e0 + static_cast<int>(threadIdx.x); e < e1; e += blockDim.x) {
    T s = 0;
    for (int c0 = 0; c0 < nclusters; c0 += 8) {   // 8 loads in flight, summed in cluster order
      T v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = (c0 + u < nclusters) ? __ldcg(cpart + static_cast<int64_t>(c0 + u) * count + e) : T(0);
#pragma unroll
      for (int u = 0; u < 8; ++u) s += v[u];
    }
    out[e] = s;
  }
  __threadfence();
  cl.sync();
  if (rank == 0 && threadIdx.x == 0) *ticket = 0;   // ready for the next launch
  return true;
}

// Second level over independent groups (e.g. column tiles): true in the one CTA that calls last.
__device__ __forceinline__ bool last_of(unsigned* ticket, unsigned total, int* flag_sm) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned old = atomicAdd(ticket, 1u);
    const int last = (old == total - 1) ? 1 : 0;
    if (last) *ticket = 0;
    *flag_sm = last;
  }
  __syncthreads();
  const int last = *flag_sm;
  if (last) __threadfence();
  return last != 0;
}

}  // namespace frsvt
