// TMA stage kernel: the same tile arithmetic as stage_kernel, with the tile
// loads issued as tensor-memory-accelerator copies (cp.async.bulk.tensor)
// into a ring of shared-memory tile buffers, so the next tiles are in flight
// while the current one is transformed. Completion is tracked by one
// mbarrier per buffer (expect-tx bytes, phase parity).
//
// Shared-memory layouts written by the copies (both 128-byte swizzled, both
// read without bank conflicts by 16 pencils x 2 neighbouring indices):
//  * row side (the transform axis is contiguous in HBM): boxes of 16 indices
//    x 16 pencils; box c holds indices 16c..16c+15, one 128-byte row per
//    pencil -- see rowbox_index().
//  * column side (16 consecutive pencils are contiguous in HBM): boxes of 32
//    indices; one 128-byte row of 16 pencils per index -- the swz() layout.
#pragma once
#include <cuda.h>

#include "gbfft_device.cuh"

namespace gbfft {

constexpr int kRowBoxBytes = kRowBoxN * kTileP * 8;
constexpr int kColBoxBytes = kColBoxN * kTileP * 8;

enum TmaSrc : int { kTmaRow = 1, kTmaCol = 2 };

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for phase `parity` of the barrier, giving up after `limit_ns`.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity, long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  unsigned long long t0;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t0));
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    if ((long long)(t - t0) > limit_ns) return false;
  }
}

// 4D tiled tensor copy global -> shared, completing on `bar`.
__device__ __forceinline__ void tma_load_4d(void* smem_dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tma_prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ------------------------------------------------------ tile geometry

// Threads and resident blocks of the TMA kernel. Long pencils (512) get one
// 1024-thread block per SM (one butterfly per thread per radix-8 pass) so 32
// warps hide the arithmetic latency while the copies stream; length 256 gets
// three blocks per SM (with 8-row column boxes its two-buffer ring fits), shorter
// pencils two.
__host__ __device__ constexpr int tma_threads(int L) {
  return L == 512 ? 1024 : (L >= 1024 ? 512 : threads_for(L));
}
__host__ __device__ constexpr int tma_blocks_per_sm(int L) { return L >= 512 ? 1 : (L == 256 ? 3 : 2); }

template <int L, int KIND, int SRC>
struct TmaGeom {
  static constexpr int n_in = KIND == kC2RPre ? L + 1 : L;
  static constexpr int rows_row = ((n_in + kRowBoxN - 1) / kRowBoxN) * kRowBoxN;
  static constexpr int rows_col = ((n_in + kColBoxN - 1) / kColBoxN) * kColBoxN;
  static constexpr int rows_min = (KIND == kR2CPost || KIND == kC2RPre) ? L + 1 : L;
  static constexpr int rows_a = SRC == kTmaRow ? rows_row : rows_col;
  static constexpr int rows_b = rows_a > rows_min ? rows_a : rows_min;
  static constexpr int rows = ((rows_b + 7) / 8) * 8;          // whole 1 KB swizzle atoms
  static constexpr int buf_bytes = rows * kTileP * 8;
  static constexpr int tw_bytes = (tw_table_len(L) + L + 1) * 8;
  // the rings of the resident blocks fit in 220 KB of the SM's 228 KB
  static constexpr int budget = 220 * 1024 / tma_blocks_per_sm(L) - 1024;
  static constexpr int nbuf = (3 * buf_bytes + tw_bytes <= budget) ? 3 : (2 * buf_bytes + tw_bytes <= budget) ? 2 : 1;
  static constexpr size_t smem = 1024 + (size_t)nbuf * buf_bytes + tw_bytes;
  static constexpr int row_boxes = (n_in + kRowBoxN - 1) / kRowBoxN;
  static constexpr int col_boxes = (n_in + kColBoxN - 1) / kColBoxN;
};

// ------------------------------------------------------------ the kernel

// Issue the copies of tile `tile` into buffer `buf`, completing on `bar`.
template <int L, int KIND, int SRC>
__device__ __forceinline__ void tma_issue_tile(const CUtensorMap* map, const StageDesc& d, long long tile,
                                               float2* buf, uint64_t* bar) {
  using G = TmaGeom<L, KIND, SRC>;
  // 32-bit decode (tile counts stay below 2^32): 64-bit division is a subroutine call
  const unsigned t32 = (unsigned)tile;
  const unsigned gc = t32 % (unsigned)d.n_gchunks;
  const unsigned rest = t32 / (unsigned)d.n_gchunks;
  const int o = (int)(rest % (unsigned)d.n_outer);
  const int b = (int)(rest / (unsigned)d.n_outer);
  const int g0 = (int)gc * kTileP;
  char* dst = reinterpret_cast<char*>(buf);
  if constexpr (SRC == kTmaRow) {
    mbar_arrive_expect_tx(bar, (unsigned)(G::row_boxes * kRowBoxBytes));
    for (int c = 0; c < G::row_boxes; ++c) tma_load_4d(dst + c * kRowBoxBytes, map, 32 * c, g0, o, b, bar);
  } else {
    mbar_arrive_expect_tx(bar, (unsigned)(G::col_boxes * kColBoxBytes));
    for (int j = 0; j < G::col_boxes; ++j)
      tma_load_4d(dst + j * kColBoxBytes, map, 2 * g0, kColBoxN * j, o, b, bar);
  }
}

// Tile arithmetic on a buffer the copies filled (input already in shared
// memory, in the row-box or the swizzled column layout).
template <int L, int DIR, int KIND, int SRC, int THREADS>
__device__ __forceinline__ void process_tile_tma(const StageDesc& d, long long tile, float2* sm, const float2* tw,
                                                 const float2* tw2) {
  int o, g0;
  TileIO io = make_io(d, tile, o, g0);
  const bool row_out = d.out_mode == kRow;
  constexpr int SL = SRC == kTmaRow ? 1 : 0;  // source layout of pass 0
  if constexpr (KIND == kPlain) {
    if (row_out) {
      fft_passes<L, DIR, THREADS, false, false, false, 0, SL>(sm, tw, io);
      row_store<THREADS, L>(sm, io);
    } else {
      fft_passes<L, DIR, THREADS, false, true, false, 0, SL>(sm, tw, io);
    }
  } else if constexpr (KIND == kR2CPost) {
    fft_passes<L, -1, THREADS, false, false, false, 0, SL>(sm, tw, io);
    if (row_out) {
      r2c_post<L, THREADS>(sm, tw2, d.interior);
      row_store<THREADS, L + 1>(sm, io);
    } else {
      r2c_post_col_store<L, THREADS>(sm, tw2, d.interior, io);
    }
  } else if constexpr (KIND == kC2RPre) {
    static_assert(SRC == kTmaCol, "the merge reads the column layout");
    c2r_pre<L, THREADS>(sm, tw2, d.interior);
    fft_passes<L, +1, THREADS, false, false, false>(sm, tw, io);
    row_store<THREADS, L>(sm, io);
  } else if constexpr (KIND == kPoissonZ) {
    TileIO io_nos = io;
    io_nos.scale = 1.f;
    fft_passes<L, -1, THREADS, false, false, false, 0, SL>(sm, tw, io_nos);
    poisson_multiply<L, THREADS>(sm, g0, o, d.pz_ny, d.scale);
    if (row_out) {
      fft_passes<L, +1, THREADS, false, false, false>(sm, tw, io_nos);
      row_store<THREADS, L>(sm, io_nos);
    } else {
      fft_passes<L, +1, THREADS, false, true, false>(sm, tw, io_nos);
    }
  }
}

// One launch per stage, one block per SM (or more for short lengths). Block
// b handles tiles b, b + grid, b + 2 grid, ...; thread 0 keeps the copies of
// the next nbuf-1 tiles in flight. Every mbarrier wait is bounded; on a
// timeout the block records kDevErrTimeout in *err and stops.
template <int L, int DIR, int KIND, int SRC>
__global__ void __launch_bounds__(tma_threads(L), tma_blocks_per_sm(L))
    tma_stage_kernel(const __grid_constant__ CUtensorMap map, StageDesc d, int* err, long long timeout_ns) {
  using G = TmaGeom<L, KIND, SRC>;
  constexpr int THREADS = tma_threads(L);
  constexpr int NB = G::nbuf;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                         ~static_cast<uintptr_t>(1023));
  float2* bufs = reinterpret_cast<float2*>(base);
  float2* tw = reinterpret_cast<float2*>(base + (size_t)NB * G::buf_bytes);
  constexpr int TWL = tw_table_len(L);
  float2* tw2 = tw + TWL;
  __shared__ __align__(8) uint64_t full[NB];
  __shared__ int s_fail;
  const long long stride = gridDim.x;
  pdl_launch_next();
  if (threadIdx.x == 0) {
    tma_prefetch_map(&map);
    for (int i = 0; i < NB; ++i) mbar_init(&full[i], 1);
    mbar_init_fence();
    s_fail = 0;
  }
  load_twiddles<L, THREADS>(tw, tw2, d, KIND == kR2CPost || KIND == kC2RPre);
  pdl_wait_prev();  // the first copies read the previous grid's output
  if (threadIdx.x == 0) {
    for (int i = 0; i < NB; ++i) {
      const long long t = blockIdx.x + i * stride;
      if (t < d.n_tiles)
        tma_issue_tile<L, KIND, SRC>(&map, d, t, bufs + (size_t)i * (G::buf_bytes / 8), &full[i]);
    }
  }
  __syncthreads();
  long long k = 0;
  for (long long t = blockIdx.x; t < d.n_tiles; t += stride, ++k) {
    const int slot = (int)(k % NB);
    const unsigned parity = (unsigned)((k / NB) & 1);
    float2* sm = bufs + (size_t)slot * (G::buf_bytes / 8);
    const bool ok = mbar_wait_bounded(&full[slot], parity, timeout_ns);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) {
        atomicCAS(err, 0, kDevErrTimeout);
        s_fail = 1;
      }
      break;
    }
    process_tile_tma<L, DIR, KIND, SRC, THREADS>(d, t, sm, tw, tw2);
    // order this thread's shared-memory accesses of the buffer before the
    // tensor copy that will overwrite it, then free the buffer
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      const long long tn = t + NB * stride;
      if (tn < d.n_tiles) tma_issue_tile<L, KIND, SRC>(&map, d, tn, sm, &full[slot]);
    }
  }
  // after a timeout, wait (bounded) for copies still in flight before the
  // block's shared memory is released
  __syncthreads();
  if (s_fail && threadIdx.x == 0) {
    for (long long j = k; j < k + NB; ++j) {
      const long long tj = blockIdx.x + j * stride;
      if (tj >= d.n_tiles) break;
      mbar_wait_bounded(&full[(int)(j % NB)], (unsigned)((j / NB) & 1), timeout_ns);
    }
  }
}

}  // namespace gbfft
