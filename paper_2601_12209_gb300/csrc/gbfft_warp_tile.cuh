// Tile body of the warp-per-pencil stages (L = R1 x 32, R1 = 8, 16), shared
// by the warp-per-pencil stage kernels (gbfft_warp.cuh) and the persistent
// kernel (gbfft_kernels.cuh), which runs it for the stages of its launch that
// the plan selects.
#pragma once
#include "gbfft_device.cuh"

namespace gbfft {

constexpr int kWarpThreads = 32 * kTileP;  // one warp per pencil of the tile

template <int L>
struct WarpGeom {
  static constexpr int R1 = L / 32;                     // values per lane
  static constexpr int C = 32 / R1;                     // lanes per k1 in step 5
  static constexpr int kPitch = C <= 2 ? 33 : 32 + C;   // transpose buffer row pitch (float2)
  static constexpr int kBuf = R1 * kPitch;
  static constexpr int kMin = (L + 1 > kBuf ? L + 1 : kBuf);
  static constexpr int kRegion = kMin + ((17 - kMin % 16) % 16);  // smallest pitch >= kMin, = 1 mod 16
  static_assert(R1 * C == 32 && (C == 1 || C == 2 || C == 4), "L = 1024, 512 or 256");
  static_assert(kRegion % 16 == 1, "odd-by-16 region pitch");
};

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
// An unscaled stage (scale 1, every stage but a transform's last) skips the
// multiplies. FIXED (the rows -> columns launches): thread (q, n0) stores rows
// n0 + i (THREADS / 16) in whole passes (compile-time shared-memory offsets,
// one pointer step per row), then the rows left.
template <int NROWS, int RG, int THREADS = kWarpThreads, int PAD_SHIFT = 0, int PAD = 0, bool FIXED = false>
__device__ __forceinline__ void warp_col_store(const float2* sm, const TileIO& io) {
  if constexpr (FIXED) {
    constexpr int RPP = THREADS / kTileP;  // rows per pass
    constexpr int PASSES = NROWS / RPP;
    static_assert(PAD == 0 || (1 << PAD_SHIFT) % RPP == 0, "a pass stays inside one padded block");
    const int q = threadIdx.x & 15, n0 = threadIdx.x / kTileP;
    if (q < io.valid) {
      const float2* src = sm + q * RG + n0;
      float2* dst = io.gout + q + (long long)n0 * io.out_n;
      const long long step = (long long)RPP * io.out_n;
      if (io.scale == 1.f) {
#pragma unroll
        for (int i = 0; i < PASSES; ++i) {
          st_data(dst, src[i * RPP + ((i * RPP) >> PAD_SHIFT) * PAD]);
          dst += step;
        }
      } else {
#pragma unroll
        for (int i = 0; i < PASSES; ++i) {
          st_data(dst, cscale(src[i * RPP + ((i * RPP) >> PAD_SHIFT) * PAD], io.scale));
          dst += step;
        }
      }
    }
    for (int it = PASSES * RPP * kTileP + threadIdx.x; it < NROWS * kTileP; it += THREADS) {
      const int qq = it & 15, n = it >> 4;
      if (qq < io.valid)
        st_data(io.gout + qq + n * io.out_n, cscale(sm[qq * RG + n + (n >> PAD_SHIFT) * PAD], io.scale));
    }
  } else if (io.scale == 1.f) {
    for (int it = threadIdx.x; it < NROWS * kTileP; it += THREADS) {
      const int q = it & 15, n = it >> 4;
      if (q < io.valid) st_data(io.gout + q + n * io.out_n, sm[q * RG + n + (n >> PAD_SHIFT) * PAD]);
    }
  } else {
    for (int it = threadIdx.x; it < NROWS * kTileP; it += THREADS) {
      const int q = it & 15, n = it >> 4;
      if (q < io.valid) st_data(io.gout + q + n * io.out_n, cscale(sm[q * RG + n + (n >> PAD_SHIFT) * PAD], io.scale));
    }
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

// 32-point DFT of one lane's values in registers, natural order in and out:
// n = a + 4 b (a < 4, b < 8), k = k1 + 8 k2 (k1 < 8, k2 < 4):
//   X[k1 + 8 k2] = sum_a W_4^(a k2) [W_32^(a k1) sum_b x[a + 4 b] W_8^(b k1)],
// eight-point DFTs over b, the twiddles W_32^(a k1) (forward-sign table
// w32[j] = W_32^j in shared memory, conjugated for DIR = +1), four-point DFTs
// over a.
template <int DIR>
__device__ __forceinline__ void dft32(float2 (&v)[32], const float2* w32) {
  float2 t[4][8];
  static_for<4>([&](auto ac) {
    constexpr int a = decltype(ac)::value;
    static_for<8>([&](auto bc) {
      constexpr int b = decltype(bc)::value;
      t[a][b] = v[a + 4 * b];
    });
    dft8<DIR>(t[a]);
    if constexpr (a > 0) {
      static_for<7>([&](auto kc) {
        constexpr int k1 = decltype(kc)::value + 1;
        t[a][k1] = cmul(t[a][k1], tw_dir<DIR>(w32[a * k1]));
      });
    }
  });
  static_for<8>([&](auto kc) {
    constexpr int k1 = decltype(kc)::value;
    float2 u[4] = {t[0][k1], t[1][k1], t[2][k1], t[3][k1]};
    dft4<DIR>(u);
    static_for<4>([&](auto qc) {
      constexpr int k2 = decltype(qc)::value;
      v[k1 + 8 * k2] = u[k2];
    });
  });
}

template <int R, int DIR>
__device__ __forceinline__ void warp_dft(float2 (&v)[R], const float2* w32) {
  if constexpr (R == 32) dft32<DIR>(v, w32);
  else dft<R, DIR>(v);
}

// Steps 1 and 2 on lane t's values x[t + 32 i] (i < R1), then the transpose
// write: y_t[k1] lands in wr[k1 * P + t]. (warp_tile below spells these steps
// out in place: the same arithmetic, kept inline where the stage kernels run it.)
template <int L, int DIR>
__device__ __forceinline__ void warp_steps12(float2 (&v)[WarpGeom<L>::R1], float2* wr, const float2* tws,
                                             const float2* w32, int t) {
  constexpr int R1 = WarpGeom<L>::R1, P = WarpGeom<L>::kPitch;
  warp_dft<R1, DIR>(v, w32);
#pragma unroll
  for (int k = 1; k < R1; ++k) v[k] = cmul(v[k], tw_dir<DIR>(tws[k * 32 + t]));
#pragma unroll
  for (int k = 0; k < R1; ++k) wr[k * P + t] = v[k];
}

// Steps 3 to 5 from the transpose buffer wr: lane (k1, c) = (lane / C, lane % C)
// ends with X[k1 + R1 k + R1^2 m] in v[k] (k < R1; m = c for C = 2, the
// digit-reversed c for C = 4, 0 for C = 1).
template <int L, int DIR>
__device__ __forceinline__ void warp_steps345(float2 (&v)[WarpGeom<L>::R1], const float2* wr, const float2* w32) {
  using G = WarpGeom<L>;
  constexpr int R1 = G::R1, C = G::C, P = G::kPitch;
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int k1 = lane / C, c = lane % C;
#pragma unroll
  for (int a = 0; a < R1; ++a) v[a] = wr[k1 * P + C * a + c];
  warp_dft<R1, DIR>(v, w32);
#pragma unroll
  for (int k = 0; k < R1; ++k) {
    if constexpr (C == 1) {
      // length 1024: the radix-32 step above was the last level
    } else if constexpr (C == 2) {
      v[k] = cmul(v[k], tw_dir<DIR>(w32[c * R1 + k]));  // u_c = W_32^(c k) Z_c
      const float2 q = make_float2(__shfl_xor_sync(kFull, v[k].x, 1), __shfl_xor_sync(kFull, v[k].y, 1));
      v[k] = c ? csub(q, v[k]) : cadd(v[k], q);
    } else {
      v[k] = cmul(v[k], tw_dir<DIR>(w32[c * R1 + k]));  // u_c = W_32^(c k) Z_c
      // radix 4 across lanes c = c0 + 2 c1: pairs c1 = 0/1, W_4^(c0 m0), pairs c0 = 0/1
      float2 q = make_float2(__shfl_xor_sync(kFull, v[k].x, 2), __shfl_xor_sync(kFull, v[k].y, 2));
      v[k] = (c >> 1) ? csub(q, v[k]) : cadd(v[k], q);
      if (c == 3) v[k] = mul_w4<DIR>(v[k]);
      q = make_float2(__shfl_xor_sync(kFull, v[k].x, 1), __shfl_xor_sync(kFull, v[k].y, 1));
      v[k] = (c & 1) ? csub(q, v[k]) : cadd(v[k], q);
    }
  }
}

// One tile of a warp-per-pencil stage: warp p of the block's 16 owns pencil p.
// tws = W_L^(t k1) at [k1 * 32 + t] (forward sign), w32 = W_32^(c k2') at
// [c * R1 + k2'] (length 1024, C = 1: W_32^j at [j], the radix-32
// twiddles), tw2 = W_2L^k (real kinds); all in shared memory. Called by
// all kWarpThreads threads of the block; the tile's region and twiddles are
// the caller's.
// Layout of a warp-per-pencil launch: IO = 2 in_mode + out_mode (kRow 0, kCol 1)
// fixes the two sides at compile time, so a kernel holds only its own load and
// store paths; IO = -1 reads them from the descriptor (the persistent kernel).
__host__ __device__ constexpr int warp_io(int in_mode, int out_mode) { return 2 * in_mode + out_mode; }

template <int L, int DIR, int KIND, int IO = -1>
__device__ __forceinline__ void warp_tile(const StageDesc& d, long long tile, float2* sm, const float2* tws,
                                          const float2* w32, const float2* tw2) {
  using G = WarpGeom<L>;
  constexpr int R1 = G::R1, C = G::C, P = G::kPitch, RG = G::kRegion;
  constexpr unsigned kFull = 0xffffffffu;
  const int lane = threadIdx.x & 31, p = threadIdx.x >> 5;
  const int k1 = lane / C, c = lane % C;
  const int m = C == 2 ? c : ((c >> 1) + 2 * (c & 1));  // output block of this lane after step 5
  float2* wr = sm + p * RG;                               // this warp's pencil region
  const bool row_in = IO < 0 ? d.in_mode == kRow : (IO >> 1) == kRow;
  const bool row_out = IO < 0 ? d.out_mode == kRow : (IO & 1) == kRow;
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
      // lane t of warp p: x[t + 32 i] of pencil p (coalesced along the row; a row side has element
      // stride 1, which the rows -> columns launches spell out as immediate offsets)
      const float2* src = io.gin + row_pencil(d, g0, p, io.in_g);
      if (IO == warp_io(kRow, kCol) && io.in_n == 1) {
        src += lane;
#pragma unroll
        for (int i = 0; i < R1; ++i) v[i] = (p < io.valid) ? ld_data(src + 32 * i) : make_float2(0.f, 0.f);
      } else {
#pragma unroll
        for (int i = 0; i < R1; ++i)
          v[i] = (p < io.valid) ? ld_data(src + (lane + 32 * i) * io.in_n) : make_float2(0.f, 0.f);
      }
    }
    warp_dft<R1, DIR>(v, w32);
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
    warp_dft<R1, DIR>(v, w32);
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
  warp_dft<R1, DIR>(v, w32);
#pragma unroll
  for (int k = 0; k < R1; ++k) {
    if constexpr (C == 1) {
      // length 1024: the radix-32 step above was the last level
    } else if constexpr (C == 2) {
      v[k] = cmul(v[k], tw_dir<DIR>(w32[c * R1 + k]));  // u_c = W_32^(c k) Z_c
      const float2 q = make_float2(__shfl_xor_sync(kFull, v[k].x, 1), __shfl_xor_sync(kFull, v[k].y, 1));
      v[k] = c ? csub(q, v[k]) : cadd(v[k], q);
    } else {
      v[k] = cmul(v[k], tw_dir<DIR>(w32[c * R1 + k]));  // u_c = W_32^(c k) Z_c
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
      if (io.scale != 1.f) {
#pragma unroll
        for (int k = 0; k < R1; ++k) v[k] = cscale(v[k], io.scale);
      }
#pragma unroll
      for (int k = 0; k < R1; ++k) st_data(dst + (k1 + R1 * k + R1 * R1 * m) * io.out_n, v[k]);
    }
    if (!row_in) __syncthreads();  // the next column-side tile writes every warp's region
    else __syncwarp();             // this warp's region is reused by the next tile
  } else {
    __syncwarp();  // every lane has read the transpose buffer
    // the lanes of one half-warp differ in k1 and m; each block of R1^2
    // elements is shifted by 16 / C slots so that they hit distinct banks
    constexpr int kPadShift = R1 == 32 ? 10 : (R1 == 16 ? 8 : 6), kPad = C == 1 ? 0 : 16 / C;
    static_assert(R1 * R1 == (1 << kPadShift), "R1^2 elements per output block");
    static_assert(L + (C - 1) * kPad <= RG, "padded pencil fits its region");
#pragma unroll
    for (int k = 0; k < R1; ++k) wr[k1 + R1 * k + R1 * R1 * m + m * kPad] = v[k];
    __syncthreads();
    warp_col_store<L, RG, kWarpThreads, kPadShift, kPad, IO >= 0 && (IO & 1) == kCol>(sm, io);
    __syncthreads();
  }
}

// Twiddle tables of a warp-per-pencil stage (natural twiddles d.twn in global
// memory): tws[k1 * 32 + t] = W_L^(t k1), w32[c * R1 + k2'] = W_L^(R1 c k2').
template <int L, int THREADS>
__device__ __forceinline__ void warp_load_twiddles(float2* tws, float2* w32, const StageDesc& d) {
  constexpr int R1 = WarpGeom<L>::R1;
  for (int i = threadIdx.x; i < L; i += THREADS) tws[i] = d.twn[(i & 31) * (i >> 5)];
  if (threadIdx.x < 32)
    w32[threadIdx.x] = R1 == 32 ? d.twn[(L / 32) * threadIdx.x]  // W_32^j
                                : d.twn[(R1 * (threadIdx.x / R1) * (threadIdx.x % R1)) % L];
}

}  // namespace gbfft
