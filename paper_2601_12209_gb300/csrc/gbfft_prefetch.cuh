// C2R x stage with the next tile's column-side input prefetched by cp.async.
//
// The inverse x stage of a real transform (Section IV-A's mirrored sequence,
// last step) reads the half spectrum on the column side: bins k = 0..M of 16
// consecutive pencils, one 128-byte line per bin, and merges each pair of bins
// (k, M-k) into rows k and M-k of the length-M complex transform whose
// output is the real row (the C2R identities of c2r_merge_pair). The
// thread-load kernel issues those loads into registers right before the
// merge, so each tile waits for one HBM latency with little else in flight.
//
// Here the block keeps a second shared-memory buffer, `raw`, for the raw bins
// of its NEXT tile. Right after this tile's merge has consumed `raw`, every
// thread issues 16-byte cp.async copies (global -> shared, no registers held)
// of the next tile's lines, then runs this tile's passes and row store while
// they are in flight. At the next iteration the block waits for its copies,
// merges from shared memory, and repeats. Tiles that are ragged or not
// 16-byte addressable (pair_vec_ok false) take the synchronous fused load.
#pragma once
#include "gbfft_kernels.cuh"

namespace gbfft {

struct PrefetchKernel {
  int L;
  const void* fn;
  int threads;
  size_t smem;
};

std::vector<PrefetchKernel>& prefetch_registry();

// raw[k][c]: bin k of pencil pair c (16 bytes), chunk index XOR-ed with k mod 8
__device__ __forceinline__ int raw_index(int k, int c) { return (k << 3) | (c ^ (k & 7)); }

template <int M>
constexpr size_t prefetch_smem_bytes() {
  // tile [M+1][16], raw [M+1][8] float4, twiddles, W_2M^k
  return sizeof(float2) * ((size_t)(M + 1) * kTileP) + sizeof(float4) * ((size_t)(M + 1) * 8) +
         sizeof(float2) * ((size_t)tw_table_len(M) + (M + 1));
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Issue the copies of bins 0..M of the tile's 16 pencils (8 pencil pairs per bin).
template <int M, int THREADS>
__device__ __forceinline__ void c2r_prefetch_issue(float4* raw, const TileIO& io) {
  const float4* g = reinterpret_cast<const float4*>(io.gin);
  const long long row = io.in_n >> 1;  // float4 per bin
  for (int it = threadIdx.x; it < (M + 1) * 8; it += THREADS) {
    const int k = it >> 3, c = it & 7;
    cp_async16(raw + raw_index(k, c), g + (long long)k * row + c);
  }
  cp_async_commit();
}

// Merge the bins held in raw into the tile (same arithmetic as the fused column load).
template <int M, int THREADS, bool UNIT>
__device__ __forceinline__ void c2r_merge_from_raw_impl(float2* sm, const float4* raw, const float2* tw2,
                                                        float interior) {
  constexpr int NPAIR = M / 2 + 1;
  for (int it = threadIdx.x; it < NPAIR * 8; it += THREADS) {
    const int k = it >> 3, c = it & 7;
    const float4 a = raw[raw_index(k, c)];
    const float4 b = raw[raw_index(M - k, c)];  // k = 0: row M; 2k = M: row k again
    c2r_merge_pair_to<M, UNIT>(sm, tw2, interior, it, a, b);
  }
}

template <int M, int THREADS>
__device__ __forceinline__ void c2r_merge_from_raw(float2* sm, const float4* raw, const float2* tw2, float interior) {
  if (interior == 1.f) c2r_merge_from_raw_impl<M, THREADS, true>(sm, raw, tw2, interior);
  else c2r_merge_from_raw_impl<M, THREADS, false>(sm, raw, tw2, interior);
}

// Blocks per SM: the tile and the raw buffer take 2 x 33 KB at M = 256 (three
// blocks fit), 2 x 66 KB at M = 512 (one).
__host__ __device__ constexpr int prefetch_min_blocks(int M) { return M >= 512 ? 1 : 3; }

template <int M>
__global__ void __launch_bounds__(threads_for(M), prefetch_min_blocks(M)) c2r_prefetch_kernel(StageDesc d) {
  constexpr int THREADS = threads_for(M);
  extern __shared__ float4 smem4[];
  float2* sm = reinterpret_cast<float2*>(smem4);
  float4* raw = smem4 + (M + 1) * kTileP / 2;
  float2* tw = reinterpret_cast<float2*>(raw + (M + 1) * 8);
  constexpr int TWL = tw_table_len(M);
  float2* tw2 = tw + TWL;
  pdl_launch_next();
  load_twiddles<M, THREADS>(tw, tw2, d, true);
  __syncthreads();
  pdl_wait_prev();
  int o, g0;
  long long tile = blockIdx.x;
  if (tile < d.n_tiles) {
    const TileIO io = make_io(d, tile, o, g0);
    if (pair_vec_ok(io.gin, io.in_n, io.valid)) c2r_prefetch_issue<M, THREADS>(raw, io);
  }
  for (; tile < d.n_tiles; tile += gridDim.x) {
    const TileIO io = make_io(d, tile, o, g0);
    if (pair_vec_ok(io.gin, io.in_n, io.valid)) {
      cp_async_wait_all();
      __syncthreads();  // every thread's copies have landed
      c2r_merge_from_raw<M, THREADS>(sm, raw, tw2, d.interior);
      __syncthreads();  // raw consumed, tile complete
    } else {
      col_load_c2r_pre<M, THREADS>(sm, tw2, d.interior, io);
    }
    const long long next = tile + gridDim.x;
    if (next < d.n_tiles) {
      const TileIO nio = make_io(d, next, o, g0);
      if (pair_vec_ok(nio.gin, nio.in_n, nio.valid)) c2r_prefetch_issue<M, THREADS>(raw, nio);
    }
    fft_passes<M, +1, THREADS, false, false, false>(sm, tw, io);
    row_store<THREADS, M, THREADS == M>(sm, io);
    __syncthreads();
  }
  cp_async_wait_all();
}

template <int M>
PrefetchKernel make_prefetch_entry() {
  return PrefetchKernel{M, reinterpret_cast<const void*>(&c2r_prefetch_kernel<M>), threads_for(M),
                        prefetch_smem_bytes<M>()};
}

}  // namespace gbfft
