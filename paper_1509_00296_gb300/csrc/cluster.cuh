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
  const int per = (count + 4 * CL - 1) / (4 * CL) * 4;   // multiples of 4 (float4 columns)
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
  if constexpr (sizeof(T) == 4) {
    if ((count & 3) == 0 && (e0 & 3) == 0) {
      // float4 columns; the clusters split into H interleaved groups summed by different
      // threads (all loads of a group in flight), the H group sums then added in group order
      // through part_sm (no longer read by the cluster): one L2 round trip instead of one per
      // eight clusters.
      const int nv = (e1 - e0) / 4;
      int H = nv > 0 ? static_cast<int>(blockDim.x) / nv : 1;
      H = H < 1 ? 1 : (H > CL ? CL : H);
      if (nv > 0 && H * nv > count / 4) H = (count / 4) / nv;   // red[] stays inside part_sm
      if (H < 1) H = 1;
      float4* red = reinterpret_cast<float4*>(part_sm);
      const int t = static_cast<int>(threadIdx.x);
      for (int w = t; w < nv * H; w += blockDim.x) {
        const int j = w % nv, h = w / nv;
        const float4* src = reinterpret_cast<const float4*>(cpart) + (e0 / 4 + j);
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int c0 = h; c0 < nclusters; c0 += 16 * H) {          // 16 loads in flight per thread
          float4 v[16];
#pragma unroll
          for (int u = 0; u < 16; ++u)
            v[u] = (c0 + u * H < nclusters) ? __ldcg(src + static_cast<int64_t>(c0 + u * H) * (count / 4))
                                            : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            acc.x += v[u].x;
            acc.y += v[u].y;
            acc.z += v[u].z;
            acc.w += v[u].w;
          }
        }
        red[h * nv + j] = acc;
      }
      __syncthreads();
      for (int j = t; j < nv; j += blockDim.x) {
        float4 s4 = red[j];
        for (int h = 1; h < H; ++h) {
          const float4 v = red[h * nv + j];
          s4.x += v.x;
          s4.y += v.y;
          s4.z += v.z;
          s4.w += v.w;
        }
        reinterpret_cast<float4*>(out)[e0 / 4 + j] = s4;
      }
    } else {
      for (int e = e0 + static_cast<int>(threadIdx.x); e < e1; e += blockDim.x) {
        T s = 0;
        for (int c0 = 0; c0 < nclusters; ++c0) s += __ldcg(cpart + static_cast<int64_t>(c0) * count + e);
        out[e] = s;
      }
    }
  } else {
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
  }
  cl.sync();                                   // the cluster barrier publishes out to the cluster
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
