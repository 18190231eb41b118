// Length-512 stage with one warp per pencil.
//
// The Stockham stage kernel exchanges every pass through the shared tile
// (three passes of radix 8 at length 512: six shared-memory round trips and
// seven block barriers per tile). Here each of the 16 warps of a block owns
// one pencil of the tile and factors 512 = 16 x 32 (the four-step split of
// the 1D FFT into a radix-16 and a radix-32 level, Section III-A's per-axis
// transform):
//   n = t + 32 i (lane t holds x[t + 32 i], i < 16), k = k1 + 16 k2:
//   1. y_t[k1] = sum_i x[t + 32 i] W16^(i k1)             (registers)
//   2. y_t[k1] *= W512^(t k1)                              (twiddles)
//   3. transpose through a per-warp buffer: lane (k1, b) takes
//      z[a] = y_(2a + b)[k1], a < 16                       (no block barrier)
//   4. Z_b[k2'] = sum_a z[a] W16^(a k2')                   (registers)
//   5. X[k1 + 16 k2'] = Z_0 + W32^k2' Z_1, X[k1 + 16 (k2' + 16)] = Z_0 - W32^k2' Z_1
//      with the partner lane (b ^ 1) by shuffles.
// Row-side pencils are read and written by their warp directly (coalesced
// along the row); column-side input or output goes through the shared tile
// once (the pack / unpack of the redistribution): a column-side input is read
// with lanes along the pencils (lane (tb, q) of warp w takes t = 2w + tb of
// pencil q), step 1 runs in that layout, and step 3 gathers pencil q into
// warp q's region; a column-side output is written by each warp into its own
// region and stored with lanes along the pencils. Regions are pencil-major
// (pitch 529 float2: the 16 pencils of one element fall in 16 different bank
// pairs) and hold the warp's transpose buffer too.
#pragma once
#include "gbfft_kernels.cuh"

namespace gbfft {

constexpr int kWarpL = 512;
constexpr int kWarpThreads = 32 * kTileP;  // one warp per pencil of the tile
constexpr int kWarpPitch = 33;             // row pitch (float2) of the per-warp transpose buffer
constexpr int kWarpRegion = 529;           // float2 per warp: one pencil (512) or the 16 x 33 buffer (528), + 1
static_assert(kWarpRegion >= kWarpL && kWarpRegion >= 16 * kWarpPitch && kWarpRegion % 16 == 1,
              "a warp region holds a pencil and the transpose buffer; odd pitch spreads banks");

struct WarpKernel {
  int L, dir;
  const void* fn;
  int threads;
  size_t smem;
};

std::vector<WarpKernel>& warp_registry();

constexpr size_t warp_smem_bytes() { return sizeof(float2) * ((size_t)kTileP * kWarpRegion + kWarpL + 16); }

// Column-side store of the pencil-major tile: lanes run along the 16 pencils
// of one element (one 128-byte line of global memory).
__device__ __forceinline__ void warp_col_store(const float2* sm, const TileIO& io) {
  for (int it = threadIdx.x; it < kWarpL * kTileP; it += kWarpThreads) {
    const int p = it & 15, n = it >> 4;
    if (p < io.valid) st_data(io.gout + p + n * io.out_n, cscale(sm[p * kWarpRegion + n], io.scale));
  }
}

template <int DIR>
__global__ void __launch_bounds__(kWarpThreads, 2) warp_stage_kernel(StageDesc d) {
  constexpr unsigned kFull = 0xffffffffu;
  extern __shared__ float4 smem4[];
  float2* sm = reinterpret_cast<float2*>(smem4);
  float2* tws = sm + kTileP * kWarpRegion;  // [k1][t] = W512^(t k1), forward sign
  float2* w32 = tws + kWarpL;               // W32^k2 = W512^(16 k2)
  for (int i = threadIdx.x; i < kWarpL; i += kWarpThreads) tws[i] = d.twn[(i & 31) * (i >> 5)];
  if (threadIdx.x < 16) w32[threadIdx.x] = d.twn[16 * threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, p = threadIdx.x >> 5;
  const int k1 = lane >> 1, b = lane & 1;
  float2* wr = sm + p * kWarpRegion;  // this warp's pencil / transpose buffer
  const bool row_in = d.in_mode == kRow, row_out = d.out_mode == kRow;
  for (long long tile = blockIdx.x; tile < d.n_tiles; tile += gridDim.x) {
    int o, g0;
    const TileIO io = make_io(d, tile, o, g0);
    float2 v[16];
    if (row_in) {
      // lane t of warp p: x[t + 32 i] of pencil p (coalesced along the row)
      const float2* src = io.gin + p * io.in_g;
#pragma unroll
      for (int i = 0; i < 16; ++i)
        v[i] = (p < io.valid) ? ld_data(src + (lane + 32 * i) * io.in_n) : make_float2(0.f, 0.f);
      dft<16, DIR>(v);
#pragma unroll
      for (int k = 1; k < 16; ++k) v[k] = cmul(v[k], tw_dir<DIR>(tws[k * 32 + lane]));
#pragma unroll
      for (int k = 0; k < 16; ++k) wr[k * kWarpPitch + lane] = v[k];
      __syncwarp();
    } else {
      // column side: lane (tb, q) of warp w takes t = 2w + tb of pencil q, so
      // the 16 lanes of a half-warp read one 128-byte line; step 1 then runs
      // in this layout and the result goes to pencil q's region
      const int pq = lane & 15, t = 2 * p + (lane >> 4);
      const float2* src = io.gin + pq;
#pragma unroll
      for (int i = 0; i < 16; ++i)
        v[i] = (pq < io.valid) ? ld_data(src + (t + 32 * i) * io.in_n) : make_float2(0.f, 0.f);
      dft<16, DIR>(v);
#pragma unroll
      for (int k = 1; k < 16; ++k) v[k] = cmul(v[k], tw_dir<DIR>(tws[k * 32 + t]));
      float2* rq = sm + pq * kWarpRegion;
#pragma unroll
      for (int k = 0; k < 16; ++k) rq[k * kWarpPitch + t] = v[k];
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 16; ++a) v[a] = wr[k1 * kWarpPitch + 2 * a + b];
    dft<16, DIR>(v);
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const float2 q = make_float2(__shfl_xor_sync(kFull, v[k].x, 1), __shfl_xor_sync(kFull, v[k].y, 1));
      const float2 wo = cmul(tw_dir<DIR>(w32[k]), b ? v[k] : q);  // W32^k Z_1
      const float2 e = b ? q : v[k];                                 // Z_0
      v[k] = b ? csub(e, wo) : cadd(e, wo);
    }
    // lane (k1, b) holds X[k1 + 16 k + 256 b], k < 16
    if (row_out) {
      if (p < io.valid) {
        float2* dst = io.gout + p * io.out_g;
#pragma unroll
        for (int k = 0; k < 16; ++k) st_data(dst + (k1 + 16 * k + 256 * b) * io.out_n, cscale(v[k], io.scale));
      }
      if (!row_in) __syncthreads();  // the next column-side tile writes every warp's region
      else __syncwarp();             // this warp's buffer is reused by the next tile
    } else {
      __syncwarp();  // every lane has read the transpose buffer
#pragma unroll
      for (int k = 0; k < 16; ++k) wr[k1 + 16 * k + 256 * b] = v[k];
      __syncthreads();
      warp_col_store(sm, io);
      __syncthreads();
    }
  }
}

template <int DIR>
WarpKernel make_warp_entry() {
  return WarpKernel{kWarpL, DIR, reinterpret_cast<const void*>(&warp_stage_kernel<DIR>), kWarpThreads,
                    warp_smem_bytes()};
}

}  // namespace gbfft
