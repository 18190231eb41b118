// Stage kernels with one warp per pencil, lengths L = 32 R1 (R1 = 8, 16).
//
// The Stockham stage kernel exchanges every pass through the shared tile (at
// length 512, three radix-8 passes: six shared-memory round trips and seven
// block barriers per tile). Here each of the 16 warps of a block owns one
// pencil of the tile and splits the length-L transform into two levels
// (Section III-A's per-axis 1D FFT, written as the four-step split
// L = R1 x 32), with C = 32 / R1:
//   n = t + 32 i (lane t holds x[t + 32 i], i < R1), k = k1 + R1 k2 (k2 < 32):
//   1. y_t[k1] = sum_i x[t + 32 i] W_R1^(i k1)                   (registers)
//   2. y_t[k1] *= W_L^(t k1)                                     (twiddles)
//   3. transpose through the warp's buffer: lane (k1, c) takes
//      z[a] = y_(C a + c)[k1], a < R1                            (no block barrier)
//   4. Z_c[k2'] = sum_a z[a] W_R1^(a k2')                        (registers)
//   5. X[k1 + R1 (k2' + R1 m)] = sum_c W_C^(c m) W_32^(c k2') Z_c[k2'],
//      a radix-C transform across the C lanes of (k1, .) by shuffles.
// Row-side pencils are read and written by their warp directly (coalesced
// along the row). A column-side input is read with lanes along the pencils
// (lane (tb, q) of warp w takes t = 2w + tb of pencil q), step 1 runs in that
// layout, and step 3 gathers pencil q into warp q's region; a column-side
// output is written by each warp into its region and stored with lanes along
// the pencils. The real-data kinds run their split (R2C) or merge (C2R) on
// the warp's region, next to the transform. Regions are pencil-major with an
// odd-by-16 pitch, so the 16 pencils of one element fall in 16 bank pairs.
#pragma once
#include "gbfft_kernels.cuh"

namespace gbfft {

constexpr int kWarpThreads = 32 * kTileP;  // one warp per pencil of the tile

template <int L>
struct WarpGeom {
  static constexpr int R1 = L / 32;                     // values per lane
  static constexpr int C = 32 / R1;                     // lanes per k1 in step 5
  static constexpr int kPitch = C == 2 ? 33 : 32 + C;   // transpose buffer row pitch (float2)
  static constexpr int kBuf = R1 * kPitch;
  static constexpr int kMin = (L + 1 > kBuf ? L + 1 : kBuf);
  static constexpr int kRegion = kMin + ((17 - kMin % 16) % 16);  // smallest pitch >= kMin, = 1 mod 16
  static_assert(R1 * C == 32 && (C == 2 || C == 4), "L = 512 or 256");
  static_assert(kRegion % 16 == 1, "odd-by-16 region pitch");
};

struct WarpKernel {
  int L, dir, kind;
  const void* fn;
  int threads;
  size_t smem;
};

std::vector<WarpKernel>& warp_registry();

template <int L>
constexpr size_t warp_smem_bytes() {
  // regions, W_L^(t k1) [k1][t], W_32^(c k2') [c][k2'], W_2L^k (real kinds)
  return sizeof(float2) * ((size_t)kTileP * WarpGeom<L>::kRegion + L + 32 + (L + 1));
}

// R2C split of one pencil held in natural order in `r` (rows 0..M): the same
// identities as r2c_post, bins 1..M-1 scaled by `interior`.
template <int M>
__device__ __forceinline__ void warp_r2c_post(float2* r, const float2* tw2, float interior) {
  const int lane = threadIdx.x & 31;
  for (int k = lane; k <= M / 2; k += 32) {
    if (k == 0) {
      const float2 z0 = r[0];
      r[0] = make_float2(z0.x + z0.y, 0.f);
      r[M] = make_float2(z0.x - z0.y, 0.f);
    } else if (2 * k < M) {
      const float2 A = r[k], B = r[M - k];
      const float2 ze = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));
      const float2 zo = make_float2(0.5f * (A.y + B.y), -0.5f * (A.x - B.x));
      const float2 t = cmul(tw2[k], zo);
      r[k] = cscale(cadd(ze, t), interior);
      r[M - k] = cscale(cconj(csub(ze, t)), interior);
    } else {
      r[k] = cscale(cconj(r[k]), interior);
    }
  }
}

// C2R merge of one pencil (rows 0..M in, rows 0..M-1 out): the identities of
// c2r_pre, with the Hermitian projection of bins 0 and M.
template <int M>
__device__ __forceinline__ void warp_c2r_pre(float2* r, const float2* tw2, float interior) {
  const int lane = threadIdx.x & 31;
  for (int k = lane; k <= M / 2; k += 32) {
    if (k == 0) {
      const float a = r[0].x, c = r[M].x;
      r[0] = make_float2(a + c, a - c);
    } else if (2 * k < M) {
      const float2 xk = cscale(r[k], interior), xm = cscale(r[M - k], interior);
      const float2 e = make_float2(xk.x + xm.x, xk.y - xm.y);
      const float2 dd = make_float2(xk.x - xm.x, xk.y + xm.y);
      const float2 o = cmul(dd, cconj(tw2[k]));
      r[k] = make_float2(e.x - o.y, e.y + o.x);
      r[M - k] = make_float2(e.x + o.y, -e.y + o.x);
    } else {
      const float2 xk = cscale(r[k], interior);
      r[k] = make_float2(2.f * xk.x, -2.f * xk.y);
    }
  }
}

// multiply by W_4 = exp(DIR 2 pi i / 4) = DIR * i
template <int DIR>
__device__ __forceinline__ float2 mul_w4(float2 a) {
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

// Column-side store of rows 0..NROWS-1 of the pencil-major tile: lanes run
// along the 16 pencils of one element (one 128-byte line of global memory).
template <int NROWS, int RG>
__device__ __forceinline__ void warp_col_store(const float2* sm, const TileIO& io) {
  for (int it = threadIdx.x; it < NROWS * kTileP; it += kWarpThreads) {
    const int q = it & 15, n = it >> 4;
    if (q < io.valid) st_data(io.gout + q + n * io.out_n, cscale(sm[q * RG + n], io.scale));
  }
}

// Length 256 keeps 8 values per lane: three blocks per SM fit its registers.
template <int L, int DIR, int KIND>
__global__ void __launch_bounds__(kWarpThreads, L == 256 ? 3 : 2) warp_stage_kernel(StageDesc d) {
  using G = WarpGeom<L>;
  constexpr int R1 = G::R1, C = G::C, P = G::kPitch, RG = G::kRegion;
  constexpr unsigned kFull = 0xffffffffu;
  constexpr bool kReal = KIND == kR2CPost || KIND == kC2RPre;
  extern __shared__ float4 smem4[];
  float2* sm = reinterpret_cast<float2*>(smem4);
  float2* tws = sm + kTileP * RG;  // [k1][t] = W_L^(t k1), forward sign
  float2* w32 = tws + L;           // [c][k2'] = W_32^(c k2') = W_L^(R1 c k2')
  float2* tw2 = w32 + 32;          // W_2L^k, k <= L (real kinds)
  pdl_launch_next();
  for (int i = threadIdx.x; i < L; i += kWarpThreads) tws[i] = d.twn[(i & 31) * (i >> 5)];
  if (threadIdx.x < 32) w32[threadIdx.x] = d.twn[(R1 * (threadIdx.x / R1) * (threadIdx.x % R1)) % L];
  if constexpr (kReal)
    for (int i = threadIdx.x; i <= L; i += kWarpThreads) tw2[i] = d.tw2[i];
  __syncthreads();
  pdl_wait_prev();
  const int lane = threadIdx.x & 31, p = threadIdx.x >> 5;
  const int k1 = lane / C, c = lane % C;
  const int m = C == 2 ? c : ((c >> 1) + 2 * (c & 1));  // output block of this lane after step 5
  float2* wr = sm + p * RG;                               // this warp's pencil region
  const bool row_in = d.in_mode == kRow, row_out = d.out_mode == kRow;
  for (long long tile = blockIdx.x; tile < d.n_tiles; tile += gridDim.x) {
    int o, g0;
    const TileIO io = make_io(d, tile, o, g0);
    float2 v[R1];
    // ---- input, steps 1 and 2: y_t[k1] lands in wr[k1 * P + t] of the pencil's warp
    if (KIND == kC2RPre || row_in) {
      if constexpr (KIND == kC2RPre) {
        // the merge needs the pencil's L + 1 bins in its region first
        if (row_in) {
          for (int n = lane; n <= L; n += 32)
            wr[n] = (p < io.valid) ? ld_data(io.gin + p * io.in_g + n * io.in_n) : make_float2(0.f, 0.f);
          __syncwarp();
        } else {
          for (int it = threadIdx.x; it < (L + 1) * kTileP; it += kWarpThreads) {
            const int q = it & 15, n = it >> 4;
            sm[q * RG + n] = (q < io.valid) ? ld_data(io.gin + q + n * io.in_n) : make_float2(0.f, 0.f);
          }
          __syncthreads();
        }
        warp_c2r_pre<L>(wr, tw2, d.interior);
        __syncwarp();
#pragma unroll
        for (int i = 0; i < R1; ++i) v[i] = wr[lane + 32 * i];
        __syncwarp();  // the transpose buffer overwrites the pencil
      } else {
        // lane t of warp p: x[t + 32 i] of pencil p (coalesced along the row)
        const float2* src = io.gin + p * io.in_g;
#pragma unroll
        for (int i = 0; i < R1; ++i)
          v[i] = (p < io.valid) ? ld_data(src + (lane + 32 * i) * io.in_n) : make_float2(0.f, 0.f);
      }
      dft<R1, DIR>(v);
#pragma unroll
      for (int k = 1; k < R1; ++k) v[k] = cmul(v[k], tw_dir<DIR>(tws[k * 32 + lane]));
#pragma unroll
      for (int k = 0; k < R1; ++k) wr[k * P + lane] = v[k];
      __syncwarp();
    } else {
      // column side: lane (tb, q) of warp w takes t = 2w + tb of pencil q, so the
      // 16 lanes of a half-warp read one 128-byte line; step 1 runs in this layout
      const int pq = lane & 15, t = 2 * p + (lane >> 4);
      const float2* src = io.gin + pq;
#pragma unroll
      for (int i = 0; i < R1; ++i)
        v[i] = (pq < io.valid) ? ld_data(src + (t + 32 * i) * io.in_n) : make_float2(0.f, 0.f);
      dft<R1, DIR>(v);
#pragma unroll
      for (int k = 1; k < R1; ++k) v[k] = cmul(v[k], tw_dir<DIR>(tws[k * 32 + t]));
      float2* rq = sm + pq * RG;
#pragma unroll
      for (int k = 0; k < R1; ++k) rq[k * P + t] = v[k];
      __syncthreads();
    }
    // ---- steps 3 to 5
#pragma unroll
    for (int a = 0; a < R1; ++a) v[a] = wr[k1 * P + C * a + c];
    dft<R1, DIR>(v);
#pragma unroll
    for (int k = 0; k < R1; ++k) {
      v[k] = cmul(v[k], tw_dir<DIR>(w32[c * R1 + k]));  // u_c = W_32^(c k) Z_c
      if constexpr (C == 2) {
        const float2 q = make_float2(__shfl_xor_sync(kFull, v[k].x, 1), __shfl_xor_sync(kFull, v[k].y, 1));
        v[k] = c ? csub(q, v[k]) : cadd(v[k], q);
      } else {
        // radix 4 across lanes c = c0 + 2 c1: pairs c1 = 0/1, W_4^(c0 m0), pairs c0 = 0/1
        float2 q = make_float2(__shfl_xor_sync(kFull, v[k].x, 2), __shfl_xor_sync(kFull, v[k].y, 2));
        v[k] = (c >> 1) ? csub(q, v[k]) : cadd(v[k], q);
        if (c == 3) v[k] = mul_w4<DIR>(v[k]);
        q = make_float2(__shfl_xor_sync(kFull, v[k].x, 1), __shfl_xor_sync(kFull, v[k].y, 1));
        v[k] = (c & 1) ? csub(q, v[k]) : cadd(v[k], q);
      }
    }
    // lane (k1, c) holds X[k1 + R1 k + R1^2 m], k < R1
    if constexpr (KIND == kR2CPost) {
      __syncwarp();  // every lane has read the transpose buffer
#pragma unroll
      for (int k = 0; k < R1; ++k) wr[k1 + R1 * k + R1 * R1 * m] = v[k];
      __syncwarp();
      warp_r2c_post<L>(wr, tw2, d.interior);
      __syncwarp();
      if (row_out) {
        for (int n = lane; n <= L; n += 32)
          if (p < io.valid) st_data(io.gout + p * io.out_g + n * io.out_n, cscale(wr[n], io.scale));
        __syncwarp();
      } else {
        __syncthreads();
        warp_col_store<L + 1, RG>(sm, io);
        __syncthreads();
      }
    } else if (row_out) {
      if (p < io.valid) {
        float2* dst = io.gout + p * io.out_g;
#pragma unroll
        for (int k = 0; k < R1; ++k) st_data(dst + (k1 + R1 * k + R1 * R1 * m) * io.out_n, cscale(v[k], io.scale));
      }
      if (!row_in) __syncthreads();  // the next column-side tile writes every warp's region
      else __syncwarp();             // this warp's region is reused by the next tile
    } else {
      __syncwarp();  // every lane has read the transpose buffer
#pragma unroll
      for (int k = 0; k < R1; ++k) wr[k1 + R1 * k + R1 * R1 * m] = v[k];
      __syncthreads();
      warp_col_store<L, RG>(sm, io);
      __syncthreads();
    }
  }
}

template <int L, int DIR, int KIND>
WarpKernel make_warp_entry() {
  return WarpKernel{L, DIR, KIND, reinterpret_cast<const void*>(&warp_stage_kernel<L, DIR, KIND>), kWarpThreads,
                    warp_smem_bytes<L>()};
}

}  // namespace gbfft
