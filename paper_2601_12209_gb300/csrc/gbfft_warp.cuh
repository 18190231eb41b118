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
// Element n of a pencil sits at n + (n >> PAD_SHIFT) * PAD of its region.
template <int NROWS, int RG, int THREADS = kWarpThreads, int PAD_SHIFT = 0, int PAD = 0>
__device__ __forceinline__ void warp_col_store(const float2* sm, const TileIO& io) {
  for (int it = threadIdx.x; it < NROWS * kTileP; it += THREADS) {
    const int q = it & 15, n = it >> 4;
    if (q < io.valid) st_data(io.gout + q + n * io.out_n, cscale(sm[q * RG + n + (n >> PAD_SHIFT) * PAD], io.scale));
  }
}

// Offset of pencil p of the tile on a row side: p * stride_g, or, for a merged
// descriptor (m_split > 0), the split of m = g0 + p into (m / m_split, m % m_split).
__device__ __forceinline__ long long row_pencil(const StageDesc& d, int g0, int p, long long stride_g) {
  if (d.m_split == 0) return (long long)p * stride_g;
  const unsigned m = (unsigned)(g0 + p);
  const unsigned o = m / (unsigned)d.m_split;
  return (long long)o * d.split_o + (long long)(m - o * (unsigned)d.m_split) * d.split_g;
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
            wr[n] = (p < io.valid) ? ld_data(io.gin + row_pencil(d, g0, p, io.in_g) + n * io.in_n)
                                   : make_float2(0.f, 0.f);
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
        const float2* src = io.gin + row_pencil(d, g0, p, io.in_g);
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
          if (p < io.valid) st_data(io.gout + row_pencil(d, g0, p, io.out_g) + n * io.out_n, cscale(wr[n], io.scale));
        __syncwarp();
      } else {
        __syncthreads();
        warp_col_store<L + 1, RG>(sm, io);
        __syncthreads();
      }
    } else if (row_out) {
      if (p < io.valid) {
        float2* dst = io.gout + row_pencil(d, g0, p, io.out_g);
#pragma unroll
        for (int k = 0; k < R1; ++k) st_data(dst + (k1 + R1 * k + R1 * R1 * m) * io.out_n, cscale(v[k], io.scale));
      }
      if (!row_in) __syncthreads();  // the next column-side tile writes every warp's region
      else __syncwarp();             // this warp's region is reused by the next tile
    } else {
      __syncwarp();  // every lane has read the transpose buffer
      // the lanes of one half-warp differ in k1 and m; each block of R1^2
      // elements is shifted by 16 / C slots so that they hit distinct banks
      constexpr int kPadShift = R1 == 16 ? 8 : 6, kPad = 16 / C;
      static_assert(R1 * R1 == (1 << kPadShift), "R1^2 elements per output block");
      static_assert(L + (C - 1) * kPad <= RG, "padded pencil fits its region");
#pragma unroll
      for (int k = 0; k < R1; ++k) wr[k1 + R1 * k + R1 * R1 * m + m * kPad] = v[k];
      __syncthreads();
      warp_col_store<L, RG, kWarpThreads, kPadShift, kPad>(sm, io);
      __syncthreads();
    }
  }
}

template <int L, int DIR, int KIND>
WarpKernel make_warp_entry() {
  return WarpKernel{L, DIR, KIND, reinterpret_cast<const void*>(&warp_stage_kernel<L, DIR, KIND>), kWarpThreads,
                    warp_smem_bytes<L>()};
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
  return WarpKernel{L2 / 2, DIR, DIR < 0 ? kR2CPost : kC2RPre,
                    reinterpret_cast<const void*>(&pair_stage_kernel<L2, DIR>), kPairThreads,
                    pair_smem_bytes<L2>()};
}

}  // namespace gbfft
