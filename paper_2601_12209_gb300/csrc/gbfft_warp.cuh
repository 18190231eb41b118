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
// once (the pack / unpack of the redistribution).
#pragma once
#include "gbfft_kernels.cuh"

namespace gbfft {

constexpr int kWarpL = 512;
constexpr int kWarpThreads = 32 * kTileP;  // one warp per pencil of the tile
constexpr int kWarpPitch = 33;             // row pitch (float2) of the per-warp transpose buffer
// tile [512][16] for column-side I/O and the 16 per-warp buffers share one region
constexpr int kWarpRegion = (kTileP * 16 * kWarpPitch > kWarpL * kTileP) ? kTileP * 16 * kWarpPitch : kWarpL * kTileP;

struct WarpKernel {
  int L, dir;
  const void* fn;
  int threads;
  size_t smem;
};

std::vector<WarpKernel>& warp_registry();

constexpr size_t warp_smem_bytes() { return sizeof(float2) * ((size_t)kWarpRegion + kWarpL + 16); }

template <int DIR>
__global__ void __launch_bounds__(kWarpThreads, 2) warp_stage_kernel(StageDesc d) {
  constexpr unsigned kFull = 0xffffffffu;
  extern __shared__ float4 smem4[];
  float2* sm = reinterpret_cast<float2*>(smem4);
  float2* tws = sm + kWarpRegion;  // [k1][t] = W512^(t k1), forward sign
  float2* w32 = tws + kWarpL;      // W32^k2 = W512^(16 k2)
  for (int i = threadIdx.x; i < kWarpL; i += kWarpThreads) tws[i] = d.twn[(i & 31) * (i >> 5)];
  if (threadIdx.x < 16) w32[threadIdx.x] = d.twn[16 * threadIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, p = threadIdx.x >> 5;
  const int k1 = lane >> 1, b = lane & 1;
  float2* wb = sm + p * (16 * kWarpPitch);
  const bool row_in = d.in_mode == kRow, row_out = d.out_mode == kRow;
  for (long long tile = blockIdx.x; tile < d.n_tiles; tile += gridDim.x) {
    int o, g0;
    const TileIO io = make_io(d, tile, o, g0);
    float2 v[16];
    if (row_in) {
      const float2* src = io.gin + p * io.in_g;
#pragma unroll
      for (int i = 0; i < 16; ++i)
        v[i] = (p < io.valid) ? ld_data(src + (lane + 32 * i) * io.in_n) : make_float2(0.f, 0.f);
    } else {
      col_load<kWarpThreads, kWarpL>(sm, io);
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = sm[swz(lane + 32 * i, p)];
      __syncthreads();  // the per-warp buffers overwrite the tile
    }
    dft<16, DIR>(v);
#pragma unroll
    for (int k = 1; k < 16; ++k) v[k] = cmul(v[k], tw_dir<DIR>(tws[k * 32 + lane]));
#pragma unroll
    for (int k = 0; k < 16; ++k) wb[k * kWarpPitch + lane] = v[k];
    __syncwarp();
#pragma unroll
    for (int a = 0; a < 16; ++a) v[a] = wb[k1 * kWarpPitch + 2 * a + b];
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
      __syncwarp();  // this warp's buffer is reused by the next tile
    } else {
      __syncthreads();  // every warp is done with its buffer
#pragma unroll
      for (int k = 0; k < 16; ++k) sm[swz(k1 + 16 * k + 256 * b, p)] = v[k];
      __syncthreads();
      col_store<kWarpThreads, kWarpL>(sm, io);
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
