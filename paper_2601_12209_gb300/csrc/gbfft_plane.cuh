// Fused in-plane stages of the slab variant: one launch for the two stages
// that work inside an xy-plane.
//
// Section III-A's slab decomposition does a local 2D transform on each
// z-slab, one transpose, then the 1D transforms along z. On one GPU the 2D
// transform is the x stage and the y stage of a plane. Run as two
// grid-wide launches, the first stage's output (the whole array) leaves L2
// before the second stage reads it, so the pair moves the array through HBM
// twice. Here a thread-block cluster owns one plane: its CTAs run the first
// stage's tiles of the plane, meet at a cluster barrier (release/acquire at
// cluster scope orders the global writes before the reads), then run the
// second stage's tiles. The planes in flight across the GPU hold tens of MB,
// well inside the 129 MB L2, so the second stage reads the first stage's
// output from L2 and writes its result over it in place: one HBM read of the
// input and one write of the result for both stages.
#pragma once
#include "gbfft_kernels.cuh"

namespace gbfft {

struct PlaneKernel {
  int L1, dir1, kind1;  // first in-plane stage
  int L2, dir2, kind2;  // second in-plane stage
  const void* fn;
  int threads;
  size_t smem;
};

std::vector<PlaneKernel>& plane_registry();

__device__ __forceinline__ unsigned cluster_cta_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ unsigned cluster_cta_count() {
  unsigned n;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(n));
  return n;
}

// every thread of every CTA of the cluster arrives once, then waits
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__host__ __device__ constexpr int imax(int a, int b) { return a > b ? a : b; }

template <int L1, int L2>
__host__ __device__ constexpr int plane_threads() {
  return imax(threads_for(L1), threads_for(L2));
}

template <int L1, int L2>
__host__ __device__ constexpr int plane_min_blocks() {
  return min_blocks_for(imax(L1, L2));
}

template <int L1, int L2>
constexpr size_t plane_smem_bytes() {
  constexpr int LM = imax(L1, L2);
  return sizeof(float2) * ((size_t)(LM + 1) * kTileP + imax(tw_table_len(L1), tw_table_len(L2)) + (LM + 1));
}

// Cluster c of the grid owns plane c (batch entry and outer index of both
// stages: tile t of a stage is plane * n_gchunks + gc). CTA r of the cluster
// takes the group chunks r, r + ncta, ... of each stage.
template <int L1, int DIR1, int KIND1, int L2, int DIR2, int KIND2>
__global__ void __launch_bounds__(plane_threads<L1, L2>(), plane_min_blocks<L1, L2>())
    plane_kernel(StageDesc s1, StageDesc s2) {
  constexpr int THREADS = plane_threads<L1, L2>();
  constexpr int LM = imax(L1, L2);
  extern __shared__ float4 smem4[];
  float2* sm = reinterpret_cast<float2*>(smem4);
  float2* tw = sm + (LM + 1) * kTileP;
  float2* tw2 = tw + imax(tw_table_len(L1), tw_table_len(L2));
  const int rank = (int)cluster_cta_rank(), ncta = (int)cluster_cta_count();
  const long long plane = blockIdx.x / ncta;
  load_twiddles<L1, THREADS>(tw, tw2, s1, KIND1 == kR2CPost || KIND1 == kC2RPre);
  __syncthreads();
  for (int gc = rank; gc < s1.n_gchunks; gc += ncta) {
    process_tile<L1, DIR1, KIND1, THREADS>(s1, plane * s1.n_gchunks + gc, sm, tw, tw2);
    __syncthreads();
  }
  __threadfence();
  cluster_barrier();
  load_twiddles<L2, THREADS>(tw, tw2, s2, KIND2 == kR2CPost || KIND2 == kC2RPre);
  __syncthreads();
  for (int gc = rank; gc < s2.n_gchunks; gc += ncta) {
    process_tile<L2, DIR2, KIND2, THREADS>(s2, plane * s2.n_gchunks + gc, sm, tw, tw2);
    __syncthreads();
  }
}

template <int L1, int DIR1, int KIND1, int L2, int DIR2, int KIND2>
PlaneKernel make_plane_entry() {
  return PlaneKernel{L1, DIR1, KIND1, L2, DIR2, KIND2,
                     reinterpret_cast<const void*>(&plane_kernel<L1, DIR1, KIND1, L2, DIR2, KIND2>),
                     plane_threads<L1, L2>(), plane_smem_bytes<L1, L2>()};
}

}  // namespace gbfft
