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
#include "gbfft_warp_tile.cuh"

namespace gbfft {

struct WarpKernel {
  int L, dir, kind;
  int io;  // warp_io(in_mode, out_mode) the kernel is specialised for, -1 = any
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

// Length 256 keeps 8 values per lane: three blocks per SM fit its registers;
// length 1024 keeps 32 per lane and its 16 regions take 135 KB: one block.
__host__ __device__ constexpr int warp_min_blocks(int L) { return L == 256 ? 3 : (L == 1024 ? 1 : 2); }

template <int L, int DIR, int KIND, int IO>
__global__ void __launch_bounds__(kWarpThreads, warp_min_blocks(L)) warp_stage_kernel(StageDesc d) {
  using G = WarpGeom<L>;
  constexpr int RG = G::kRegion;
  constexpr bool kReal = KIND == kR2CPost || KIND == kC2RPre;
  extern __shared__ float4 smem4[];
  float2* sm = reinterpret_cast<float2*>(smem4);
  float2* tws = sm + kTileP * RG;  // [k1][t] = W_L^(t k1), forward sign
  float2* w32 = tws + L;           // [c][k2'] = W_32^(c k2') = W_L^(R1 c k2')
  float2* tw2 = w32 + 32;          // W_2L^k, k <= L (real kinds)
  pdl_launch_next();
  warp_load_twiddles<L, kWarpThreads>(tws, w32, d);
  if constexpr (kReal)
    for (int i = threadIdx.x; i <= L; i += kWarpThreads) tw2[i] = d.tw2[i];
  __syncthreads();
  pdl_wait_prev();
  for (long long tile = blockIdx.x; tile < d.n_tiles; tile += gridDim.x)
    warp_tile<L, DIR, KIND, IO>(d, tile, sm, tws, w32, tw2);
}

template <int L, int DIR, int KIND, int IO = -1>
WarpKernel make_warp_entry() {
  return WarpKernel{L, DIR, KIND, IO, reinterpret_cast<const void*>(&warp_stage_kernel<L, DIR, KIND, IO>),
                    kWarpThreads, warp_smem_bytes<L>()};
}

// ----------------------------------------------- two-for-one real x stages
//
// The real x stages of a length-2L real row (R2C split after, C2R merge
// before a length-L complex FFT in the Stockham kernels) run here as one
// length-2L complex FFT per PAIR of rows: z = x_p + i x_(p+1). Its transform
// Z gives both half spectra, X_p[k] = (Z[k] + conj Z[2L-k]) / 2 and
// X_(p+1)[k] = (Z[k] - conj Z[2L-k]) / 2i (k = 0..L); backwards, with the
// Hermitian extension X[2L-k] = conj X[k] (and only the real parts of bins 0
// and L, the C2R projection), Z = X_p + i X_(p+1) transforms to
// x_p + i x_(p+1). One warp per pair, 8 warps per block (a 16-pencil tile);
// the length-2L FFT is the warp kernel's two-level split. The half spectra sit
// in a pencil-major tile of pitch L + 1 (= 1 mod 16) that does not overlap the
// warps' transpose buffers.
constexpr int kPairThreads = 32 * kTileP / 2;

template <int L2>
constexpr size_t pair_smem_bytes() {
  // 8 warp regions, the 16-pencil half-spectrum tile, W_L2^(t k1), W_32^(c k2')
  return sizeof(float2) * ((size_t)(kTileP / 2) * WarpGeom<L2>::kRegion + (size_t)kTileP * (L2 / 2 + 1) + L2 + 32);
}

template <int L2, int DIR>
__global__ void __launch_bounds__(kPairThreads, 3) pair_stage_kernel(StageDesc d) {
  using G = WarpGeom<L2>;
  constexpr int R1 = G::R1, C = G::C, P = G::kPitch, RG = G::kRegion;
  constexpr int M = L2 / 2;   // half-spectrum bins 0..M
  constexpr int RO = M + 1;   // tile pitch per pencil
  static_assert(C == 2 && RO % 16 == 1, "length-512 rows: a 16 x 32 split, tile pitch 257");
  constexpr unsigned kFull = 0xffffffffu;
  extern __shared__ float4 smem4[];
  float2* sm = reinterpret_cast<float2*>(smem4);
  float2* tile = sm + (kTileP / 2) * RG;  // [pencil][k], k <= M
  float2* tws = tile + kTileP * RO;        // [k1][t] = W_L2^(t k1), forward sign
  float2* w32 = tws + L2;                  // [c][k2'] = W_32^(c k2')
  pdl_launch_next();
  for (int i = threadIdx.x; i < L2; i += kPairThreads) tws[i] = d.twn[(i & 31) * (i >> 5)];
  if (threadIdx.x < 32) w32[threadIdx.x] = d.twn[(R1 * (threadIdx.x / R1) * (threadIdx.x % R1)) % L2];
  __syncthreads();
  pdl_wait_prev();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int k1 = lane / C, c = lane % C;
  const int p0 = 2 * w, p1 = 2 * w + 1;  // the warp's pencil pair
  float2* wr = sm + w * RG;
  const bool row_in = d.in_mode == kRow, row_out = d.out_mode == kRow;
  for (long long tl = blockIdx.x; tl < d.n_tiles; tl += gridDim.x) {
    int o, g0;
    const TileIO io = make_io(d, tl, o, g0);
    float2 v[R1];
    if constexpr (DIR < 0) {
      // z[n] = x_p0[n] + i x_p1[n], lane t holding n = t + 32 i (real rows, coalesced)
      const float* g = reinterpret_cast<const float*>(io.gin);
      const float* r0 = g + 2 * p0 * io.in_g;
      const float* r1 = g + 2 * p1 * io.in_g;
#pragma unroll
      for (int i = 0; i < R1; ++i) {
        const int n = lane + 32 * i;
        v[i] = make_float2(p0 < io.valid ? __ldcg(r0 + n) : 0.f, p1 < io.valid ? __ldcg(r1 + n) : 0.f);
      }
    } else {
      // half spectra of the tile (interior bins scaled, bins 0 and M real), then Z = X_p0 + i X_p1
      for (int it = threadIdx.x; it < RO * kTileP; it += kPairThreads) {
        int q, k;
        if (row_in) {
          k = it % RO;
          q = it / RO;
        } else {
          q = it & 15;
          k = it >> 4;
        }
        float2 a = (q < io.valid) ? ld_data(io.gin + q * io.in_g + k * io.in_n) : make_float2(0.f, 0.f);
        if (k == 0 || k == M) a.y = 0.f;
        else a = cscale(a, d.interior);
        tile[q * RO + k] = a;
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < R1; ++i) {
        const int n = lane + 32 * i;
        const bool lo = n <= M;
        const int kk = lo ? n : L2 - n;
        float2 a = tile[p0 * RO + kk], b = tile[p1 * RO + kk];
        if (!lo) {
          a.y = -a.y;
          b.y = -b.y;
        }
        v[i] = make_float2(a.x - b.y, a.y + b.x);
      }
    }
    // steps 1 to 5 of the length-L2 transform (see warp_stage_kernel)
    dft<R1, DIR>(v);
#pragma unroll
    for (int k = 1; k < R1; ++k) v[k] = cmul(v[k], tw_dir<DIR>(tws[k * 32 + lane]));
#pragma unroll
    for (int k = 0; k < R1; ++k) wr[k * P + lane] = v[k];
    __syncwarp();
#pragma unroll
    for (int a = 0; a < R1; ++a) v[a] = wr[k1 * P + C * a + c];
    dft<R1, DIR>(v);
#pragma unroll
    for (int k = 0; k < R1; ++k) {
      v[k] = cmul(v[k], tw_dir<DIR>(w32[c * R1 + k]));
      const float2 q = make_float2(__shfl_xor_sync(kFull, v[k].x, 1), __shfl_xor_sync(kFull, v[k].y, 1));
      v[k] = c ? csub(q, v[k]) : cadd(v[k], q);
    }
    // lane (k1, c) holds the transform at n = k1 + R1 k + R1^2 c, k < R1
    if constexpr (DIR < 0) {
      __syncwarp();  // every lane has read the transpose buffer
#pragma unroll
      for (int k = 0; k < R1; ++k) wr[k1 + R1 * k + R1 * R1 * c] = v[k];
      __syncwarp();
      // split: X_p0[k] = (Z[k] + conj Z[L2-k]) / 2, X_p1[k] = (Z[k] - conj Z[L2-k]) / 2i
      for (int k = lane; k <= M; k += 32) {
        const float2 A = wr[k], B = wr[(L2 - k) & (L2 - 1)];
        float2 x0 = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));
        float2 x1 = make_float2(0.5f * (A.y + B.y), -0.5f * (A.x - B.x));
        if (k != 0 && k != M) {
          x0 = cscale(x0, d.interior);
          x1 = cscale(x1, d.interior);
        }
        if (row_out) {
          if (p0 < io.valid) st_data(io.gout + p0 * io.out_g + k * io.out_n, cscale(x0, io.scale));
          if (p1 < io.valid) st_data(io.gout + p1 * io.out_g + k * io.out_n, cscale(x1, io.scale));
        } else {
          tile[p0 * RO + k] = x0;
          tile[p1 * RO + k] = x1;
        }
      }
      if (row_out) {
        __syncwarp();  // this warp's region is reused by the next tile
      } else {
        __syncthreads();
        warp_col_store<RO, RO, kPairThreads>(tile, io);
        __syncthreads();
      }
    } else {
      // x_p0 = Re z, x_p1 = Im z (row side)
      float* g = reinterpret_cast<float*>(io.gout);
      float* r0 = g + 2 * p0 * io.out_g;
      float* r1 = g + 2 * p1 * io.out_g;
      const float sc = io.scale;
#pragma unroll
      for (int k = 0; k < R1; ++k) {
        const int n = k1 + R1 * k + R1 * R1 * c;
        if (p0 < io.valid) __stcg(r0 + n, v[k].x * sc);
        if (p1 < io.valid) __stcg(r1 + n, v[k].y * sc);
      }
      __syncthreads();  // the next tile's load refills the half-spectrum tile
    }
  }
}

template <int L2, int DIR>
WarpKernel make_pair_entry() {
  // registered under the Stockham kind it replaces: length L2 / 2 complex pairs per row
  return WarpKernel{L2 / 2, DIR, DIR < 0 ? kR2CPost : kC2RPre, -1,
                    reinterpret_cast<const void*>(&pair_stage_kernel<L2, DIR>), kPairThreads,
                    pair_smem_bytes<L2>()};
}

}  // namespace gbfft
