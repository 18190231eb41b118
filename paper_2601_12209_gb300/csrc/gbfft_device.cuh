// Device code of the staged 3D FFT: radix plans, butterflies, and the tile
// processor that one stage of the paper's pencil sequence runs per pencil tile.
//
// Paper mapping (arxiv 2601.12209):
//  * Section III-A: the 3D FFT is N_y N_z length-N_x transforms, a
//    redistribution, N_x N_z length-N_y transforms, a redistribution, and
//    N_x N_y length-N_z transforms. One tile = 16 pencils of one stage.
//  * Algorithm 2 (pack -> exchange -> unpack): on one GPU the exchange is HBM
//    itself; the pack is the tile's transposed store and the unpack the next
//    stage's tile load. Both move 16 consecutive complex values (128 bytes)
//    per transform index on the strided side, so every HBM access is a full
//    128-byte line.
//  * The 1D transforms are Stockham auto-sort passes of radix 2/3/4/5/8/16
//    held in registers, with one shared-memory exchange between passes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <utility>

#include "gbfft_internal.h"

namespace gbfft {

// ------------------------------------------------------------ radix plans

struct Radices {
  int n;
  int r[12];
};

// Factor L into Stockham passes: powers of two split into as few, as even
// passes as possible from {2,4,8,16}; then one pass per factor 3 and 5.
__host__ __device__ constexpr Radices make_radices(int L) {
  Radices R{0, {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0}};
  int m = L;
  int a = 0;
  while (m % 2 == 0) {
    ++a;
    m /= 2;
  }
  if (a > 0) {
    int passes = (a + 3) / 4;
    int base = a / passes, extra = a % passes;
    for (int i = 0; i < passes; ++i) R.r[R.n++] = 1 << (base + (i < extra ? 1 : 0));
  }
  while (m % 3 == 0) {
    R.r[R.n++] = 3;
    m /= 3;
  }
  while (m % 5 == 0) {
    R.r[R.n++] = 5;
    m /= 5;
  }
  if (m != 1) R.n = -1;  // unsupported prime factor
  return R;
}

__host__ __device__ constexpr int radix_prefix(int L, int pass) {
  int ns = 1;
  for (int i = 0; i < pass; ++i) ns *= make_radices(L).r[i];
  return ns;
}

// Packed twiddle table of a length-L transform: pass i >= 1 (radix R_i,
// prefix Ns_i) owns Ns_i * R_i entries, entry k * R_i + r holding
// W_{Ns_i R_i}^{r k} = exp(-2 pi i r k / (Ns_i R_i)) (r = 0 holds 1). A
// butterfly's R_i - 1 twiddles then sit next to each other (16-byte pairs).
__host__ __device__ constexpr int tw_pass_offset(int L, int pass) {
  int off = 0;
  for (int i = 1; i < pass; ++i) off += radix_prefix(L, i) * make_radices(L).r[i];
  return off;
}
__host__ __device__ constexpr int tw_table_len(int L) {
  const int n = make_radices(L).n;
  const int t = tw_pass_offset(L, n);
  return t > 0 ? t : 1;
}

// Groups of 16 threads that share the butterflies of a pass: the largest
// power of two not above the smallest butterfly count of any pass, capped at
// 32 (512 threads).
__host__ __device__ constexpr int groups_for(int L) {
  Radices R = make_radices(L);
  int mn = L;
  for (int i = 0; i < R.n; ++i) mn = (L / R.r[i]) < mn ? (L / R.r[i]) : mn;
  // up to 32 groups (512 threads); length 1024 takes 64 (1024 threads): its
  // 16 x 1025 tile fills shared memory, so one block per SM must carry the warps
  int g = 1;
  const int cap = L >= 1024 ? 64 : 32;
  while (g * 2 <= mn && g * 2 <= cap) g *= 2;
  return g;
}

__host__ __device__ constexpr int threads_for(int L) { return 16 * groups_for(L); }

// Blocks per SM the register allocation must allow: two 512-thread blocks
// (64 registers) so one block's HBM phase overlaps the other's arithmetic;
// length 1024 runs one 1024-thread block (its tile fills shared memory).
// Mixed-radix lengths of 512 threads (640, 768, 960: radix-3/5 butterflies
// next to radix-16 ones) need more than 64 registers, so they take one block.
__host__ __device__ constexpr int min_blocks_for(int L) {
  return L >= 1024 ? 1
                   : (threads_for(L) >= 512 ? ((L & (L - 1)) ? 1 : 2) : (threads_for(L) >= 256 ? (L == 256 ? 4 : 3) : 4));
}

// ---------------------------------------------------------- complex helpers

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// multiply by s*i, s = +1 or -1
template <int S>
__device__ __forceinline__ float2 mul_si(float2 a) {
  return S > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// twiddle from the forward-sign table, conjugated for the inverse direction
template <int DIR>
__device__ __forceinline__ float2 tw_dir(float2 w) {
  return DIR < 0 ? w : make_float2(w.x, -w.y);
}

// --------------------------------------------------------------- butterflies
// In-register DFT of length R with sign DIR: y[q] = sum_r x[r] exp(DIR 2 pi i rq/R).
// Constants are cos/sin of multiples of 2 pi/R written to 20 digits.

template <int DIR>
__device__ __forceinline__ void dft2(float2* a) {
  float2 t = a[0];
  a[0] = cadd(t, a[1]);
  a[1] = csub(t, a[1]);
}

template <int DIR>
__device__ __forceinline__ void dft4(float2* a) {
  float2 t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
  float2 t2 = cadd(a[1], a[3]), t3 = mul_si<DIR>(csub(a[1], a[3]));
  a[0] = cadd(t0, t2);
  a[2] = csub(t0, t2);
  a[1] = cadd(t1, t3);
  a[3] = csub(t1, t3);
}

constexpr float kSqrtHalf = 0.70710678118654752440f;

// multiply by exp(DIR 2 pi i m/8) for m = 1, 2, 3
template <int DIR, int M>
__device__ __forceinline__ float2 w8(float2 a) {
  if constexpr (M == 0) {
    return a;
  } else if constexpr (M == 2) {
    return mul_si<DIR>(a);
  } else if constexpr (M == 1) {  // (1 + DIR i)/sqrt2
    float2 t = mul_si<DIR>(a);
    return make_float2((a.x + t.x) * kSqrtHalf, (a.y + t.y) * kSqrtHalf);
  } else {  // M == 3: (-1 + DIR i)/sqrt2
    float2 t = mul_si<DIR>(a);
    return make_float2((t.x - a.x) * kSqrtHalf, (t.y - a.y) * kSqrtHalf);
  }
}

// radix-8 as radix-2 then two radix-4: X[2q] = DFT4(a_r + a_{r+4}),
// X[2q+1] = DFT4((a_r - a_{r+4}) w8^r).
template <int DIR>
__device__ __forceinline__ void dft8(float2* a) {
  float2 e[4], o[4];
  e[0] = cadd(a[0], a[4]);
  o[0] = csub(a[0], a[4]);
  e[1] = cadd(a[1], a[5]);
  o[1] = w8<DIR, 1>(csub(a[1], a[5]));
  e[2] = cadd(a[2], a[6]);
  o[2] = w8<DIR, 2>(csub(a[2], a[6]));
  e[3] = cadd(a[3], a[7]);
  o[3] = w8<DIR, 3>(csub(a[3], a[7]));
  dft4<DIR>(e);
  dft4<DIR>(o);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    a[2 * q] = e[q];
    a[2 * q + 1] = o[q];
  }
}

// cos and sin of 2 pi m / 16, m = 1..3
constexpr float kC16_1 = 0.92387953251128675613f;
constexpr float kS16_1 = 0.38268343236508977173f;

// multiply by exp(DIR 2 pi i m/16), m in [0, 8)
template <int DIR, int M>
__device__ __forceinline__ float2 w16(float2 a) {
  if constexpr (M % 2 == 0) {
    return w8<DIR, M / 2>(a);
  } else {
    // exp(DIR i theta) with theta = 2 pi M / 16
    constexpr float c = (M == 1) ? kC16_1 : (M == 3) ? kS16_1 : (M == 5) ? -kS16_1 : -kC16_1;
    constexpr float s = (M == 1) ? kS16_1 : (M == 3) ? kC16_1 : (M == 5) ? kC16_1 : kS16_1;
    constexpr float sd = DIR < 0 ? -s : s;
    return make_float2(fmaf(a.x, c, -a.y * sd), fmaf(a.x, sd, a.y * c));
  }
}

// radix-16 as radix-2 then two radix-8.
template <int DIR>
__device__ __forceinline__ void dft16(float2* a) {
  float2 e[8], o[8];
  e[0] = cadd(a[0], a[8]);
  o[0] = csub(a[0], a[8]);
  e[1] = cadd(a[1], a[9]);
  o[1] = w16<DIR, 1>(csub(a[1], a[9]));
  e[2] = cadd(a[2], a[10]);
  o[2] = w16<DIR, 2>(csub(a[2], a[10]));
  e[3] = cadd(a[3], a[11]);
  o[3] = w16<DIR, 3>(csub(a[3], a[11]));
  e[4] = cadd(a[4], a[12]);
  o[4] = w16<DIR, 4>(csub(a[4], a[12]));
  e[5] = cadd(a[5], a[13]);
  o[5] = w16<DIR, 5>(csub(a[5], a[13]));
  e[6] = cadd(a[6], a[14]);
  o[6] = w16<DIR, 6>(csub(a[6], a[14]));
  e[7] = cadd(a[7], a[15]);
  o[7] = w16<DIR, 7>(csub(a[7], a[15]));
  dft8<DIR>(e);
  dft8<DIR>(o);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    a[2 * q] = e[q];
    a[2 * q + 1] = o[q];
  }
}

// radix-3: X0 = a0 + t, X1,2 = a0 - t/2 +- DIR i (sqrt3/2)(a1 - a2), t = a1 + a2
template <int DIR>
__device__ __forceinline__ void dft3(float2* a) {
  constexpr float h = 0.86602540378443864676f;  // sqrt(3)/2
  float2 t = cadd(a[1], a[2]);
  float2 u = mul_si<DIR>(cscale(csub(a[1], a[2]), h));
  float2 m = make_float2(fmaf(-0.5f, t.x, a[0].x), fmaf(-0.5f, t.y, a[0].y));
  a[0] = cadd(a[0], t);
  a[1] = cadd(m, u);
  a[2] = csub(m, u);
}

// radix-5 with t1 = a1+a4, t2 = a2+a3, d1 = a1-a4, d2 = a2-a3.
template <int DIR>
__device__ __forceinline__ void dft5(float2* a) {
  constexpr float c1 = 0.30901699437494742410f;   // cos(2 pi/5)
  constexpr float c2 = -0.80901699437494742410f;  // cos(4 pi/5)
  constexpr float s1 = 0.95105651629515357212f;   // sin(2 pi/5)
  constexpr float s2 = 0.58778525229247312917f;   // sin(4 pi/5)
  float2 t1 = cadd(a[1], a[4]), t2 = cadd(a[2], a[3]);
  float2 d1 = csub(a[1], a[4]), d2 = csub(a[2], a[3]);
  float2 a0 = a[0];
  float2 r1 = make_float2(a0.x + c1 * t1.x + c2 * t2.x, a0.y + c1 * t1.y + c2 * t2.y);
  float2 r2 = make_float2(a0.x + c2 * t1.x + c1 * t2.x, a0.y + c2 * t1.y + c1 * t2.y);
  float2 i1 = mul_si<DIR>(make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y));
  float2 i2 = mul_si<DIR>(make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y));
  a[0] = make_float2(a0.x + t1.x + t2.x, a0.y + t1.y + t2.y);
  a[1] = cadd(r1, i1);
  a[4] = csub(r1, i1);
  a[2] = cadd(r2, i2);
  a[3] = csub(r2, i2);
}

template <int R, int DIR>
__device__ __forceinline__ void dft(float2* a) {
  if constexpr (R == 2) dft2<DIR>(a);
  else if constexpr (R == 3) dft3<DIR>(a);
  else if constexpr (R == 4) dft4<DIR>(a);
  else if constexpr (R == 5) dft5<DIR>(a);
  else if constexpr (R == 8) dft8<DIR>(a);
  else if constexpr (R == 16) dft16<DIR>(a);
}

// ------------------------------------------------------------ memory helpers

// Tile layout in shared memory: element n of pencil p at n*16 + swizzled p.
// The 16 pencils of one index n form one 128-byte row; the 16-byte chunk
// (pencil pair) index is XOR-ed with n mod 8, so both "16 pencils at one n"
// and "one pencil pair over 8 consecutive n" touch every bank once.
// XOR-ing the 16-byte chunk index (p >> 1) with (n & 7) equals XOR-ing p with
// 2 (n & 7), since the mask is even and leaves bit 0 of p alone.
__device__ __forceinline__ int swz(int n, int p) { return (n << 4) + (p ^ ((n & 7) << 1)); }

__device__ __forceinline__ float2 ld_data(const float2* p) { return __ldcg(p); }
__device__ __forceinline__ void st_data(float2* p, float2 v) { __stcg(p, v); }
__device__ __forceinline__ float4 ld_data4(const float4* p) { return __ldcg(p); }
__device__ __forceinline__ void st_data4(float4* p, float4 v) { __stcg(p, v); }

struct TileIO {
  const float2* gin;
  float2* gout;
  long long in_g, in_n, out_g, out_n;
  int valid;
  float scale;
};

// Index of the thread within the team of THREADS threads that processes one
// tile. Every kernel but the batched one runs one team per block (its block
// size is THREADS, so this is threadIdx.x); the batched kernel runs several
// tiles of a short length side by side, one per team of consecutive threads.
template <int THREADS>
__device__ __forceinline__ int ttid() {
  static_assert((THREADS & (THREADS - 1)) == 0, "team sizes are powers of two");
  return (int)(threadIdx.x & (THREADS - 1));
}

// Row-side load: the transform axis is contiguous in global memory. Lanes run
// along n (coalesced), each lane moves one pencil pair as a 16-byte smem chunk.
template <int THREADS, int NROWS>
__device__ __forceinline__ void row_load(float2* sm, const TileIO& io) {
  for (int it = ttid<THREADS>(); it < NROWS * 8; it += THREADS) {
    int n = it % NROWS, pair = it / NROWS;
    int p0 = 2 * pair;
    float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
    if (p0 < io.valid) a = ld_data(io.gin + p0 * io.in_g + n);
    if (p0 + 1 < io.valid) b = ld_data(io.gin + (p0 + 1) * io.in_g + n);
    *reinterpret_cast<float4*>(sm + ((n << 4) | ((pair ^ (n & 7)) << 1))) = make_float4(a.x, a.y, b.x, b.y);
  }
}

// FIXED (a team of one thread per row, NROWS == THREADS): thread n stores the
// 8 pencil pairs of row n with one pointer step per pair.
template <int THREADS, int NROWS, bool FIXED = false>
__device__ __forceinline__ void row_store(const float2* sm, const TileIO& io) {
  const float sc = io.scale;
  const bool unit = sc == 1.f;
  if constexpr (FIXED) {
    static_assert(NROWS == THREADS, "one thread per row");
    const int n = ttid<THREADS>();
    float2* g = io.gout + n;
    const long long step = 2 * io.out_g;
#pragma unroll
    for (int pair = 0; pair < 8; ++pair) {
      float4 v = *reinterpret_cast<const float4*>(sm + ((n << 4) | ((pair ^ (n & 7)) << 1)));
      if (!unit) v = make_float4(v.x * sc, v.y * sc, v.z * sc, v.w * sc);
      if (2 * pair < io.valid) st_data(g, make_float2(v.x, v.y));
      if (2 * pair + 1 < io.valid) st_data(g + io.out_g, make_float2(v.z, v.w));
      g += step;
    }
    return;
  }
  for (int it = ttid<THREADS>(); it < NROWS * 8; it += THREADS) {
    int n = it % NROWS, pair = it / NROWS;
    int p0 = 2 * pair;
    float4 v = *reinterpret_cast<const float4*>(sm + ((n << 4) | ((pair ^ (n & 7)) << 1)));
    if (!unit) v = make_float4(v.x * sc, v.y * sc, v.z * sc, v.w * sc);
    if (p0 < io.valid) st_data(io.gout + p0 * io.out_g + n, make_float2(v.x, v.y));
    if (p0 + 1 < io.valid) st_data(io.gout + (p0 + 1) * io.out_g + n, make_float2(v.z, v.w));
  }
}

// Column-side load/store: 16 consecutive pencils are contiguous; lanes run
// along p, so 16 lanes move one 128-byte line.
template <int THREADS, int NROWS>
__device__ __forceinline__ void col_load(float2* sm, const TileIO& io) {
  for (int it = ttid<THREADS>(); it < NROWS * 16; it += THREADS) {
    int p = it & 15, n = it >> 4;
    float2 a = make_float2(0.f, 0.f);
    if (p < io.valid) a = ld_data(io.gin + p + n * io.in_n);
    sm[swz(n, p)] = a;
  }
}

template <int THREADS, int NROWS>
__device__ __forceinline__ void col_store(const float2* sm, const TileIO& io) {
  for (int it = ttid<THREADS>(); it < NROWS * 16; it += THREADS) {
    int p = it & 15, n = it >> 4;
    if (p < io.valid) {
      float2 v = sm[swz(n, p)];
      if (io.scale != 1.f) v = make_float2(v.x * io.scale, v.y * io.scale);
      st_data(io.gout + p + n * io.out_n, v);
    }
  }
}

// ---------------------------------------------------------- Stockham passes

// One Stockham pass of radix R over the 16 pencils of the tile.
// Butterfly j (0 <= j < L/R) of pencil p reads x[j + r L/R], applies the
// twiddles W_{Ns R}^{r k} (k = j mod Ns), a radix-R DFT, and writes
// y[(j - k) R + k + q Ns]. Thread (p, g) owns butterflies j = g + t*G.
//   SRC_GLOBAL: pass 0 reads the column-side input straight from HBM.
//   DST_GLOBAL: the last pass writes the column-side output straight to HBM.
// Row-side box layout written by the tensor copies (see gbfft_tma.cuh):
// index n of pencil p, 16-index boxes of 16 pencil rows, 128-byte swizzle.
__device__ __forceinline__ int rowbox_index(int n, int p) {
  return ((n >> 4) << 8) | (p << 4) | ((((n & 15) >> 1) ^ (p & 7)) << 1) | (n & 1);
}

// Compile-time loop: f(integral_constant<int, 0>) ... f(integral_constant<int, N-1>).
// The butterfly loops use it so every register array index is a constant by
// construction (with #pragma unroll alone, the compiler keeps some of these
// loops rolled inside kernels that loop over tiles, and the arrays go to
// local memory).
template <typename F, int... Is>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

template <int L, int DIR, int THREADS, int PASS, bool SRC_GLOBAL, bool DST_GLOBAL, bool SYNC_BEFORE_WRITE,
          int SRC_LAYOUT = 0>
__device__ __forceinline__ void stockham_pass(float2* sm, const float2* tw, const TileIO& io) {
  constexpr Radices RP = make_radices(L);
  constexpr int R = RP.r[PASS];
  constexpr int Ns = radix_prefix(L, PASS);
  constexpr int NB = L / R;
  constexpr int G = THREADS / 16;
  constexpr int NBT = (NB + G - 1) / G;
  constexpr int TWO = tw_pass_offset(L, PASS);  // evaluated at compile time
  const int p = ttid<THREADS>() & 15, g = ttid<THREADS>() >> 4;
  float2 v[NBT][R];
  static_for<NBT>([&](auto tc) {
    constexpr int t = decltype(tc)::value;
    const int j = g + t * G;
    if (NB % G == 0 || j < NB) {
      static_for<R>([&](auto rc) {
        constexpr int r = decltype(rc)::value;
        const int n = j + r * NB;
        if constexpr (SRC_GLOBAL) {
          v[t][r] = (p < io.valid) ? ld_data(io.gin + p + n * io.in_n) : make_float2(0.f, 0.f);
        } else if constexpr (SRC_LAYOUT == 1) {
          v[t][r] = sm[rowbox_index(n, p)];
        } else {
          v[t][r] = sm[swz(n, p)];
        }
      });
      if constexpr (Ns > 1) {
        const int k = j % Ns;
        // tw is 16-byte aligned and every offset below is even when R is even
        const float2* twp = tw + TWO + k * R;
        if constexpr (R % 2 == 0) {
          static_for<R / 2>([&](auto hc) {
            constexpr int r = 2 * decltype(hc)::value;
            const float4 w = *reinterpret_cast<const float4*>(twp + r);
            if constexpr (r > 0) v[t][r] = cmul(v[t][r], tw_dir<DIR>(make_float2(w.x, w.y)));
            v[t][r + 1] = cmul(v[t][r + 1], tw_dir<DIR>(make_float2(w.z, w.w)));
          });
        } else {
          static_for<R - 1>([&](auto rc) {
            constexpr int r = decltype(rc)::value + 1;
            v[t][r] = cmul(v[t][r], tw_dir<DIR>(twp[r]));
          });
        }
      }
      dft<R, DIR>(v[t]);
    }
  });
  if constexpr (DST_GLOBAL) {
    if constexpr (SYNC_BEFORE_WRITE) __syncthreads();
    const bool unit = io.scale == 1.f;
    const long long step = (long long)NB * io.out_n;  // last pass: Ns R = L, outputs j + q NB
    static_for<NBT>([&](auto tc) {
      constexpr int t = decltype(tc)::value;
      const int j = g + t * G;
      if ((NB % G == 0 || j < NB) && p < io.valid) {
        float2* o = io.gout + p + (long long)j * io.out_n;
        if (unit) {
          static_for<R>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            st_data(o + q * step, v[t][q]);
          });
        } else {
          static_for<R>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            st_data(o + q * step, cscale(v[t][q], io.scale));
          });
        }
      }
    });
  } else {
    if constexpr (SYNC_BEFORE_WRITE) __syncthreads();
    static_for<NBT>([&](auto tc) {
      constexpr int t = decltype(tc)::value;
      const int j = g + t * G;
      if (NB % G == 0 || j < NB) {
        const int k = j % Ns;
        const int base = (j - k) * R + k;
        static_for<R>([&](auto qc) {
          constexpr int q = decltype(qc)::value;
          sm[swz(base + q * Ns, p)] = v[t][q];
        });
      }
    });
    __syncthreads();
  }
}

// ------------------------------------ split-precision tensor-core radix 16
//
// A radix-16 Stockham pass applies the 16-point DFT matrix
// F[q][r] = exp(s 2 pi i q r / 16) (s = -1 forward, +1 inverse) to the
// twiddled inputs of every butterfly: with one column per butterfly (pencil
// p, group j), the pass is the dense product Y = F X, in real form
// Yr = Fr Xr - Fi Xi and Yi = Fi Xr + Fr Xi. Here it runs on the tensor cores
// (mma.sync m16n8k16, FP32 accumulation): each real operand a is split into a
// pair of 16-bit floats hi = rn(a), lo = rn(a - hi), and each product keeps
// the three terms hi.hi + hi.lo + lo.hi (the dropped lo.lo term is about
// 2^-22 of the operand scale with FP16, 2^-16 with BF16). Before the split,
// each column is scaled by the power of two that puts its largest component
// in [0.5, 1) (inside the FP16 range); the outputs are scaled back exactly.
// Twiddles and the data exchange stay in FP32, as in the FP32 pass.

// cos(2 pi m / 16) for m in [0, 16), from the constants of the FP32 radix 16
__device__ __forceinline__ float cos16(int m) {
  const int a = m & 7;  // cos(x + pi) = -cos x
  const int b = a <= 4 ? a : 8 - a;  // cos(pi - x) = -cos x
  float v = b == 0 ? 1.f : b == 1 ? kC16_1 : b == 2 ? kSqrtHalf : b == 3 ? kS16_1 : 0.f;
  if (a > 4) v = -v;
  return (m & 8) ? -v : v;
}

// hi/lo pairs of (a, b), packed low element first as mma operands expect
template <int PREC>
__device__ __forceinline__ void split16x2(float a, float b, uint32_t& hi, uint32_t& lo) {
  if constexpr (PREC == kPrecF16Split) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
  }
}

// D += A B for one m16n8k16 tile: A 16x16 row-major fragment, B 16x8 fragment
template <int PREC>
__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  if constexpr (PREC == kPrecF16Split) {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  } else {
    asm("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
}

// This lane's A fragments of Fr and Fi (hi and lo). Fragment register i holds
// rows q = g + 8 (i & 1), columns r = 2t + 8 (i >> 1) + {0, 1}, with
// g = lane / 4, t = lane % 4 (the m16n8k16 operand layout).
template <int PREC, int DIR>
struct Dft16Frags {
  uint32_t re_hi[4], re_lo[4], im_hi[4], im_lo[4];
  __device__ __forceinline__ Dft16Frags() {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const float sg = DIR < 0 ? -1.f : 1.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int q = g + ((i & 1) << 3);
      const int r = 2 * t + ((i >> 1) << 3);
      const int m0 = (q * r) & 15, m1 = (q * (r + 1)) & 15;
      split16x2<PREC>(cos16(m0), cos16(m1), re_hi[i], re_lo[i]);
      // sin(2 pi m / 16) = cos(2 pi (m - 4) / 16)
      split16x2<PREC>(sg * cos16((m0 + 12) & 15), sg * cos16((m1 + 12) & 15), im_hi[i], im_lo[i]);
    }
  }
};

// One column group on the tensor cores: the 8 butterflies whose inputs this
// lane holds as x[0..3] (inputs r = 2t, 2t+1, 2t+8, 2t+9 of butterfly g,
// already twiddled). y[0..7] receives outputs (q = g, pencil 2t), (q = g,
// pencil 2t+1), (q = g+8, pencil 2t), (q = g+8, pencil 2t+1) as re, im pairs.
template <int PREC, int DIR>
__device__ __forceinline__ void tc16_group(const Dft16Frags<PREC, DIR>& F, const float2 (&x)[4], float (&y)[8]) {
  constexpr unsigned kFull = 0xffffffffu;
  const int tq = threadIdx.x & 3;
  // power-of-two column scale: the 4 lanes of a column reduce their maxima
  float m = fmaxf(fmaxf(fmaxf(fabsf(x[0].x), fabsf(x[0].y)), fmaxf(fabsf(x[1].x), fabsf(x[1].y))),
                  fmaxf(fmaxf(fabsf(x[2].x), fabsf(x[2].y)), fmaxf(fabsf(x[3].x), fabsf(x[3].y))));
  m = fmaxf(m, __shfl_xor_sync(kFull, m, 1));
  m = fmaxf(m, __shfl_xor_sync(kFull, m, 2));
  int e = (int)((__float_as_uint(m) >> 23) & 0xffu);  // m in [2^(e-127), 2^(e-126))
  e = e == 0 ? 126 : min(e, 252);                      // zero or subnormal column: scale 1
  const float sc = __uint_as_float((uint32_t)(253 - e) << 23);  // 2^(126 - e)
  uint32_t rh0, rl0, rh1, rl1, ih0, il0, ih1, il1;
  split16x2<PREC>(x[0].x * sc, x[1].x * sc, rh0, rl0);
  split16x2<PREC>(x[2].x * sc, x[3].x * sc, rh1, rl1);
  split16x2<PREC>(x[0].y * sc, x[1].y * sc, ih0, il0);
  split16x2<PREC>(x[2].y * sc, x[3].y * sc, ih1, il1);
  constexpr uint32_t kNeg = 0x80008000u;  // sign bits of both 16-bit halves
  float yr[4] = {0.f, 0.f, 0.f, 0.f}, yi[4] = {0.f, 0.f, 0.f, 0.f};
  // small terms first, then hi.hi
  mma_16816<PREC>(yr, F.re_hi, rl0, rl1);
  mma_16816<PREC>(yr, F.re_lo, rh0, rh1);
  mma_16816<PREC>(yr, F.im_hi, il0 ^ kNeg, il1 ^ kNeg);
  mma_16816<PREC>(yr, F.im_lo, ih0 ^ kNeg, ih1 ^ kNeg);
  mma_16816<PREC>(yr, F.re_hi, rh0, rh1);
  mma_16816<PREC>(yr, F.im_hi, ih0 ^ kNeg, ih1 ^ kNeg);
  mma_16816<PREC>(yi, F.im_hi, rl0, rl1);
  mma_16816<PREC>(yi, F.im_lo, rh0, rh1);
  mma_16816<PREC>(yi, F.re_hi, il0, il1);
  mma_16816<PREC>(yi, F.re_lo, ih0, ih1);
  mma_16816<PREC>(yi, F.im_hi, rh0, rh1);
  mma_16816<PREC>(yi, F.re_hi, ih0, ih1);
  // output columns 2t and 2t+1 were scaled by the lanes 8t and 8t+4
  const int e0 = __shfl_sync(kFull, e, 8 * tq);
  const int e1 = __shfl_sync(kFull, e, 8 * tq + 4);
  const float s0 = __uint_as_float((uint32_t)(e0 + 1) << 23);  // 2^(e0 - 126)
  const float s1 = __uint_as_float((uint32_t)(e1 + 1) << 23);
  y[0] = yr[0] * s0;
  y[1] = yi[0] * s0;
  y[2] = yr[1] * s1;
  y[3] = yi[1] * s1;
  y[4] = yr[2] * s0;
  y[5] = yi[2] * s0;
  y[6] = yr[3] * s1;
  y[7] = yi[3] * s1;
}

// The radix-16 pass PASS of a length-L tile on the tensor cores. A warp takes
// butterfly group j for all 16 pencils: two column groups of 8 butterflies
// (pencils 8h..8h+7, h = 0, 1). Lane (g, t) loads inputs r = 2t, 2t+1, 2t+8,
// 2t+9 of butterflies (j, 8h+g) -- the m16n8k16 B layout -- and receives
// outputs q = g, g+8 of butterflies (j, 8h+2t) and (j, 8h+2t+1). Reads,
// barrier, writes as in stockham_pass.
//
// Bank spreading: when the rows a warp touches share one swizzle phase (all
// loads when L/16 is a multiple of 8, the stores when Ns is), lanes t >= 2 (for
// loads) or g >= 4 (for stores) take the other half of the tile first, so every
// access instruction splits evenly over both 16-bank halves of a 128-byte row.
template <int L, int DIR, int THREADS, int PASS, bool SRC_GLOBAL, bool DST_GLOBAL, bool SYNC_BEFORE_WRITE, int PREC>
__device__ __forceinline__ void stockham_pass_tc16(float2* sm, const float2* tw, const TileIO& io) {
  constexpr int R = 16;
  static_assert(make_radices(L).r[PASS] == R, "tensor-core pass is radix 16");
  static_assert(kTileP == 16 && THREADS % 32 == 0, "two column groups of 8 pencils per tile row");
  constexpr int Ns = radix_prefix(L, PASS);
  constexpr int NB = L / R;
  constexpr int W = THREADS / 32;
  constexpr int JT = (NB + W - 1) / W;
  constexpr int TWO = tw_pass_offset(L, PASS);
  constexpr bool kSpreadLoads = !SRC_GLOBAL && NB % 8 == 0;
  constexpr bool kSpreadStores = !DST_GLOBAL && Ns % 8 == 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int gq = lane >> 2, tq = lane & 3;
  const int hl = kSpreadLoads ? (tq >> 1) : 0;
  const int hw = kSpreadStores ? (gq >> 2) : 0;
  const Dft16Frags<PREC, DIR> F;
  float acc[JT][2][8];
  static_for<JT>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    const int j = warp + i * W;
    if (NB % W == 0 || j < NB) {
      // load k reads half (k >> 2) ^ hl, input u = k & 3
      float2 ld[8];
      static_for<8>([&](auto kc) {
        constexpr int k = decltype(kc)::value;
        constexpr int u = k & 3;
        const int p = (((k >> 2) ^ hl) << 3) + gq;
        const int n = j + (2 * tq + (u & 1) + ((u >> 1) << 3)) * NB;
        if constexpr (SRC_GLOBAL) {
          ld[k] = (p < io.valid) ? ld_data(io.gin + p + n * io.in_n) : make_float2(0.f, 0.f);
        } else {
          ld[k] = sm[swz(n, p)];
        }
      });
      float4 w0 = make_float4(1.f, 0.f, 1.f, 0.f), w1 = w0;
      if constexpr (Ns > 1) {
        // tw is 16-byte aligned and TWO + k R + 2t is even
        const float2* twp = tw + TWO + (j % Ns) * R + 2 * tq;
        w0 = *reinterpret_cast<const float4*>(twp);
        w1 = *reinterpret_cast<const float4*>(twp + 8);
      }
      static_for<2>([&](auto hc) {
        constexpr int h = decltype(hc)::value;
        float2 x[4];
        static_for<4>([&](auto uc) {
          constexpr int u = decltype(uc)::value;
          x[u] = hl ? ld[((h ^ 1) << 2) | u] : ld[(h << 2) | u];
        });
        if constexpr (Ns > 1) {
          x[0] = cmul(x[0], tw_dir<DIR>(make_float2(w0.x, w0.y)));
          x[1] = cmul(x[1], tw_dir<DIR>(make_float2(w0.z, w0.w)));
          x[2] = cmul(x[2], tw_dir<DIR>(make_float2(w1.x, w1.y)));
          x[3] = cmul(x[3], tw_dir<DIR>(make_float2(w1.z, w1.w)));
        }
        tc16_group<PREC, DIR>(F, x, acc[i][h]);
      });
    }
  });
  if constexpr (SYNC_BEFORE_WRITE) __syncthreads();
  static_for<JT>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    const int j = warp + i * W;
    if (NB % W == 0 || j < NB) {
      static_for<2>([&](auto mc) {
        constexpr int m = decltype(mc)::value;
        float a[8];
        static_for<8>([&](auto ec) {
          constexpr int e = decltype(ec)::value;
          a[e] = hw ? acc[i][m ^ 1][e] : acc[i][m][e];
        });
        const int pc = ((m ^ hw) << 3) + 2 * tq;
        if constexpr (DST_GLOBAL) {
          // last pass (Ns R = L): output q of group j is element j + q NB
          const float f = io.scale;
          static_for<4>([&](auto vc) {
            constexpr int v = decltype(vc)::value;
            const int pp = pc + (v & 1);
            const int n = j + (gq + ((v >> 1) << 3)) * NB;
            if (pp < io.valid) st_data(io.gout + pp + n * io.out_n, make_float2(a[2 * v] * f, a[2 * v + 1] * f));
          });
        } else {
          const int k = j % Ns;
          const int base = (j - k) * R + k;
          // pencils pc, pc + 1 stay adjacent under the swizzle (pc even)
          *reinterpret_cast<float4*>(sm + swz(base + gq * Ns, pc)) = make_float4(a[0], a[1], a[2], a[3]);
          *reinterpret_cast<float4*>(sm + swz(base + (gq + 8) * Ns, pc)) = make_float4(a[4], a[5], a[6], a[7]);
        }
      });
    }
  });
  if constexpr (!DST_GLOBAL) __syncthreads();
}

// ----------------------- split-precision radix 16 on the 5th-generation tensor cores
//
// The same split-operand DFT-16 products as stockham_pass_tc16, issued as
// tcgen05.mma: one thread per block issues them, the operands sit in shared
// memory and the FP32 accumulators in tensor memory. Butterfly b of the pass
// (pencil p = b mod 16, group j = b / 16; L butterflies per tile) is row b of
// an L x 32 operand A = [Re x_0..15 | Im x_0..15] (twiddled inputs scaled by
// the power of two that puts the row's largest component in [0.5, 1)), split
// into A_hi and A_lo. The real form of the DFT matrix,
//   B = [[Fr, Fi], [-Fi, Fr]] (32 x 32, row k = input, column n = output),
// so that [Yr | Yi] = [Xr | Xi] B, is split into B_hi and B_lo once per block.
// Each 128-row M-tile m of A gives D_m = A_hi B_lo + A_lo B_hi + A_hi B_hi
// (small terms first; six MMAs of M = 128, N = 32, K = 16) in tensor-memory
// columns 32 m .. 32 m + 31, row b in lane b mod 128. A block of THREADS (a
// multiple of 128) gives thread t the butterflies b = t + THREADS i; warp w may
// read lanes 32 (w mod 4) .. +31 of tensor memory, which hold b mod 128 =
// t mod 128, so every thread reads back exactly the rows it packed. While the
// MMAs run, the tile's data lives in the threads' registers, so A_hi and A_lo
// (L rows of 64 bytes each) are written over the tile, which holds L + 1 rows
// of 128 bytes.
//
// Operands are K-major with no swizzle: 8-row x 16-byte core matrices, element
// (row, k) of a 16-bit operand at byte (row / 8) * 512 + (k / 8) * 128 +
// (row mod 8) * 16 + (k mod 8) * 2 (the descriptor's leading byte offset, 128,
// steps along K; its stride byte offset, 512, along the rows).

__host__ __device__ constexpr int tc5_ncols(int L) {
  int need = 32 * (L / 128), c = 32;
  while (c < need) c *= 2;
  return c;
}

// Lengths with a 5th-generation tensor-core pass: a radix-16 pass, butterflies
// filling 128-row M-tiles, and a block of whole warpgroups.
__host__ __device__ constexpr bool tc5_capable(int L, int threads) {
  bool r16 = false;
  for (int i = 0; i < make_radices(L).n; ++i) r16 = r16 || make_radices(L).r[i] == 16;
  return r16 && L % 128 == 0 && threads % 128 == 0;
}

struct Tc5Shared {
  uint64_t mbar;      // completion of a pass's MMAs (tcgen05.commit)
  uint32_t tmem;      // tensor-memory base address of the block's accumulators
  uint32_t phase;     // parity of the next completion
  int* err;           // plan error word (a bounded wait that ran out records kDevErrTimeout)
  uint32_t pad;
  alignas(128) unsigned char b_ops[2][32 * 32 * 2];  // B_hi, B_lo in the operand layout
};

__device__ __forceinline__ Tc5Shared& tc5_shared() {
  __shared__ Tc5Shared s;
  return s;
}

__device__ __forceinline__ int tc5_off(int row, int k) {
  return ((row >> 3) << 9) + ((k >> 3) << 7) + ((row & 7) << 4) + ((k & 7) << 1);
}

__device__ __forceinline__ uint64_t tc5_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46);
}

template <int PREC>
__device__ __forceinline__ uint32_t tc5_idesc() {
  // F32 accumulate, A and B both F16 (0) or both BF16 (1), K-major, N = 32, M = 128
  constexpr uint32_t f = prec_mma_sync(PREC) == kPrecF16Split ? 0u : 1u;
  return (1u << 4) | (f << 7) | (f << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);
}

// Block prologue: B_hi / B_lo, the completion barrier, tensor memory.
template <int L, int DIR, int PREC, int THREADS>
__device__ __forceinline__ void tc5_setup(int* err) {
  Tc5Shared& c = tc5_shared();
  const int tid = threadIdx.x;
  const float sg = DIR < 0 ? -1.f : 1.f;
  for (int i = tid; i < 32 * 16; i += THREADS) {
    const int n = i >> 4, k0 = (i & 15) << 1;  // two inputs k0, k0 + 1 of output n
    float v[2];
    for (int u = 0; u < 2; ++u) {
      const int k = k0 + u, q = n & 15, r = k & 15, m = (q * r) & 15;
      const float cr = cos16(m), si = sg * cos16((m + 12) & 15);  // Fr, Fi of F[q][r]
      v[u] = n < 16 ? (k < 16 ? cr : -si) : (k < 16 ? si : cr);
    }
    uint32_t hi, lo;
    split16x2<prec_mma_sync(PREC)>(v[0], v[1], hi, lo);
    *reinterpret_cast<uint32_t*>(c.b_ops[0] + tc5_off(n, k0)) = hi;
    *reinterpret_cast<uint32_t*>(c.b_ops[1] + tc5_off(n, k0)) = lo;
  }
  if (tid == 0) {
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&c.mbar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    c.phase = 0;
    c.err = err;
  }
  if (tid < 32) {
    const uint32_t slot = (uint32_t)__cvta_generic_to_shared(&c.tmem);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(tc5_ncols(L))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Block epilogue: every tensor-memory access of the block is done; free it.
template <int L>
__device__ __forceinline__ void tc5_teardown() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tc5_shared().tmem), "r"(tc5_ncols(L))
                 : "memory");
  }
}

// Bounded wait for the completion of parity `ph` (about 2 s); false if it ran out.
__device__ __forceinline__ bool tc5_wait(uint32_t mb, uint32_t ph) {
  uint32_t done = 0;
  unsigned long long t0 = 0;
  for (int it = 0; !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(done)
        : "r"(mb), "r"(ph)
        : "memory");
    if (!done && (it & 255) == 255) {
      unsigned long long now;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
      if (t0 == 0) t0 = now;
      else if (now - t0 > 2000000000ull) return false;
    }
  }
  return true;
}

template <int L, int DIR, int THREADS, int PASS, bool SRC_GLOBAL, bool DST_GLOBAL, int PREC>
__device__ __forceinline__ void stockham_pass_tc5(float2* sm, const float2* tw, const TileIO& io) {
  constexpr int R = 16;
  static_assert(make_radices(L).r[PASS] == R, "tensor-core pass is radix 16");
  static_assert(tc5_capable(L, THREADS), "128-row M-tiles, whole warpgroups");
  constexpr int Ns = radix_prefix(L, PASS);
  constexpr int NB = L / R;
  constexpr int G = THREADS / 16;
  constexpr int NBT = (NB + G - 1) / G;
  constexpr int TWO = tw_pass_offset(L, PASS);
  constexpr int MT = L / 128;
  Tc5Shared& c = tc5_shared();
  const int tid = threadIdx.x;
  const int p = tid & 15, g = tid >> 4;
  float2 v[NBT][R];
  float sc[NBT];
  // 1. inputs of the thread's butterflies, twiddled, and their power-of-two scale
  static_for<NBT>([&](auto tc) {
    constexpr int t = decltype(tc)::value;
    const int j = g + t * G;
    sc[t] = 1.f;
    if (NB % G == 0 || j < NB) {
      static_for<R>([&](auto rc) {
        constexpr int r = decltype(rc)::value;
        const int n = j + r * NB;
        if constexpr (SRC_GLOBAL) {
          v[t][r] = (p < io.valid) ? ld_data(io.gin + p + n * io.in_n) : make_float2(0.f, 0.f);
        } else {
          v[t][r] = sm[swz(n, p)];
        }
      });
      if constexpr (Ns > 1) {
        const float2* twp = tw + TWO + (j % Ns) * R;
        static_for<R / 2>([&](auto hc) {
          constexpr int r = 2 * decltype(hc)::value;
          const float4 w = *reinterpret_cast<const float4*>(twp + r);
          if constexpr (r > 0) v[t][r] = cmul(v[t][r], tw_dir<DIR>(make_float2(w.x, w.y)));
          v[t][r + 1] = cmul(v[t][r + 1], tw_dir<DIR>(make_float2(w.z, w.w)));
        });
      }
      float m = 0.f;
      static_for<R>([&](auto rc) {
        constexpr int r = decltype(rc)::value;
        m = fmaxf(m, fmaxf(fabsf(v[t][r].x), fabsf(v[t][r].y)));
      });
      int e = (int)((__float_as_uint(m) >> 23) & 0xffu);  // m in [2^(e-127), 2^(e-126))
      e = e == 0 ? 126 : min(e, 252);                      // zero or subnormal row: scale 1
      sc[t] = __uint_as_float((uint32_t)(e + 1) << 23);    // 2^(e - 126): the output scale
      const float s_in = __uint_as_float((uint32_t)(253 - e) << 23);  // 2^(126 - e)
      static_for<R>([&](auto rc) {
        constexpr int r = decltype(rc)::value;
        v[t][r] = cscale(v[t][r], s_in);
      });
    }
  });
  __syncthreads();  // every thread has read the tile: it now takes the operands
  // 2. rows b of A_hi and A_lo (four 16-byte core-matrix rows each)
  unsigned char* a_hi = reinterpret_cast<unsigned char*>(sm);
  unsigned char* a_lo = a_hi + L * 64;
  static_for<NBT>([&](auto tc) {
    constexpr int t = decltype(tc)::value;
    const int j = g + t * G;
    if (NB % G == 0 || j < NB) {
      const int b = tid + t * THREADS;
      static_for<4>([&](auto kc) {
        constexpr int kg = decltype(kc)::value;  // 0: Re x_0..7, 1: Re x_8..15, 2: Im x_0..7, 3: Im x_8..15
        uint32_t hi[4], lo[4];
        static_for<4>([&](auto uc) {
          constexpr int u = decltype(uc)::value;
          constexpr int r0 = (kg & 1) * 8 + 2 * u;
          if constexpr (kg < 2) split16x2<prec_mma_sync(PREC)>(v[t][r0].x, v[t][r0 + 1].x, hi[u], lo[u]);
          else split16x2<prec_mma_sync(PREC)>(v[t][r0].y, v[t][r0 + 1].y, hi[u], lo[u]);
        });
        const int off = tc5_off(b, kg * 8);
        *reinterpret_cast<uint4*>(a_hi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(a_lo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      });
    }
  });
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&c.mbar);
  const uint32_t ph = c.phase;
  // 3. one thread issues the products of every M-tile, then commits them to the barrier
  if (tid == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t idesc = tc5_idesc<PREC>();
    const uint32_t sa_hi = (uint32_t)__cvta_generic_to_shared(a_hi);
    const uint32_t sa_lo = sa_hi + L * 64;
    const uint32_t sb_hi = (uint32_t)__cvta_generic_to_shared(c.b_ops[0]);
    const uint32_t sb_lo = (uint32_t)__cvta_generic_to_shared(c.b_ops[1]);
    for (int m = 0; m < MT; ++m) {
      const uint32_t d = c.tmem + 32u * (uint32_t)m;
      const uint32_t am_hi = sa_hi + (uint32_t)m * 8192u, am_lo = sa_lo + (uint32_t)m * 8192u;
      const uint32_t as[3] = {am_hi, am_lo, am_hi};
      const uint32_t bs[3] = {sb_lo, sb_hi, sb_hi};
#pragma unroll
      for (int pr = 0; pr < 3; ++pr)
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const uint64_t ad = tc5_desc(as[pr] + 256u * ks), bd = tc5_desc(bs[pr] + 256u * ks);
          const uint32_t acc = (pr | ks) ? 1u : 0u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
  }
  // 4. wait for the products; every thread reads back its own rows and writes the outputs
  const bool ok = tc5_wait(mb, ph);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok && c.err) atomicCAS(c.err, 0, kDevErrTimeout);
  const uint32_t lane_base = (uint32_t)(32 * ((tid >> 5) & 3)) << 16;
  static_for<NBT>([&](auto tc) {
    constexpr int t = decltype(tc)::value;
    const int j = g + t * G;
    if (NB % G == 0 || j < NB) {
      const int b = tid + t * THREADS;
      uint32_t y[32];
      if (ok) {
        const uint32_t ta = c.tmem + lane_base + 32u * (uint32_t)(b >> 7);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
            "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(y[0]), "=r"(y[1]), "=r"(y[2]), "=r"(y[3]), "=r"(y[4]), "=r"(y[5]), "=r"(y[6]), "=r"(y[7]),
              "=r"(y[8]), "=r"(y[9]), "=r"(y[10]), "=r"(y[11]), "=r"(y[12]), "=r"(y[13]), "=r"(y[14]), "=r"(y[15]),
              "=r"(y[16]), "=r"(y[17]), "=r"(y[18]), "=r"(y[19]), "=r"(y[20]), "=r"(y[21]), "=r"(y[22]),
              "=r"(y[23]), "=r"(y[24]), "=r"(y[25]), "=r"(y[26]), "=r"(y[27]), "=r"(y[28]), "=r"(y[29]),
              "=r"(y[30]), "=r"(y[31])
            : "r"(ta));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      } else {
        for (int u = 0; u < 32; ++u) y[u] = 0u;
      }
      const float f = sc[t];
      if constexpr (DST_GLOBAL) {
        // last pass (Ns R = L): output q of group j is element j + q NB
        if (p < io.valid) {
          float2* o = io.gout + p + (long long)j * io.out_n;
          const long long step = (long long)NB * io.out_n;
          const float fs = f * io.scale;
          static_for<R>([&](auto qc) {
            constexpr int q = decltype(qc)::value;
            st_data(o + q * step, make_float2(__uint_as_float(y[q]) * fs, __uint_as_float(y[16 + q]) * fs));
          });
        }
      } else {
        const int k = j % Ns;
        const int base = (j - k) * R + k;
        static_for<R>([&](auto qc) {
          constexpr int q = decltype(qc)::value;
          sm[swz(base + q * Ns, p)] = make_float2(__uint_as_float(y[q]) * f, __uint_as_float(y[16 + q]) * f);
        });
      }
    }
  });
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();  // outputs in the tile; every thread has read the accumulators and the parity
  if (tid == 0) c.phase = ph ^ 1u;
}

// All passes of a length-L transform. The data starts in shared memory unless
// SRC_GLOBAL, and ends in shared memory unless DST_GLOBAL.
// SRC_LAYOUT selects how pass 0 reads shared memory: 0 the swizzled column
// layout swz(), 1 the row-side box layout of the tensor copies.
template <int L, int DIR, int THREADS, bool SRC_GLOBAL, bool DST_GLOBAL, bool INPLACE_GLOBAL, int PASS = 0,
          int SRC_LAYOUT = 0, int PREC = kPrecFP32>
__device__ __forceinline__ void fft_passes(float2* sm, const float2* tw, const TileIO& io) {
  constexpr int NP = make_radices(L).n;
  if constexpr (PASS < NP) {
    constexpr bool src_g = SRC_GLOBAL && PASS == 0;
    constexpr bool dst_g = DST_GLOBAL && PASS == NP - 1;
    // before overwriting shared memory, everyone must have read it; a direct
    // global->global single pass in place also needs the barrier
    constexpr bool sync_w = (!src_g && !dst_g) || (src_g && dst_g && INPLACE_GLOBAL);
    if constexpr (prec_is_tc5(PREC) && make_radices(L).r[PASS] == 16 && (PASS > 0 || SRC_LAYOUT == 0)) {
      stockham_pass_tc5<L, DIR, THREADS, PASS, src_g, dst_g, PREC>(sm, tw, io);
    } else if constexpr (PREC != kPrecFP32 && make_radices(L).r[PASS] == 16 && (PASS > 0 || SRC_LAYOUT == 0)) {
      stockham_pass_tc16<L, DIR, THREADS, PASS, src_g, dst_g, sync_w, prec_mma_sync(PREC)>(sm, tw, io);
    } else {
      stockham_pass<L, DIR, THREADS, PASS, src_g, dst_g, sync_w, PASS == 0 ? SRC_LAYOUT : 0>(sm, tw, io);
    }
    fft_passes<L, DIR, THREADS, SRC_GLOBAL, DST_GLOBAL, INPLACE_GLOBAL, PASS + 1, SRC_LAYOUT, PREC>(sm, tw, io);
  }
}

// ---------------------------------------------------- real-transform phases

// R2C split of one pair (k, M-k), 0 < k < M/2: the length-M FFT Z of
// z[m] = x[2m] + i x[2m+1] gives X[k] = Ze[k] + W_2M^k Zo[k] with
// Ze = (Z[k] + conj Z[M-k])/2 and Zo = (Z[k] - conj Z[M-k])/(2i); X[M-k]
// follows from the same Ze, Zo. A = Z[k], B = Z[M-k], w = W_2M^k.
__device__ __forceinline__ void r2c_split_pair(float2 A, float2 B, float2 w, float2& xk, float2& xm) {
  const float2 ze = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));
  const float2 zo = make_float2(0.5f * (A.y + B.y), -0.5f * (A.x - B.x));
  const float2 t = cmul(w, zo);
  xk = cadd(ze, t);
  xm = cconj(csub(ze, t));
}

// C2R merge of one pair (k, M-k), 0 < k < M/2: with E = X[k] + conj X[M-k]
// and O = (X[k] - conj X[M-k]) conj(w), w = W_2M^k, Z[k] = E + i O and
// Z[M-k] = conj(E) + i conj(O).
__device__ __forceinline__ void c2r_merge_pair(float2 xk, float2 xm, float2 w, float2& zk, float2& zm) {
  const float2 e = make_float2(xk.x + xm.x, xk.y - xm.y);
  const float2 d = make_float2(xk.x - xm.x, xk.y + xm.y);
  const float2 o = cmul(d, cconj(w));
  zk = make_float2(e.x - o.y, e.y + o.x);
  zm = make_float2(e.x + o.y, -e.y + o.x);
}

__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 cat2(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }

// True when pencils p, p+1 (p even) of every row of the tile form one aligned
// 16-byte chunk in global memory: a full tile, an even row stride and a
// 16-byte aligned tile base.
__device__ __forceinline__ bool pair_vec_ok(const float2* base, long long row_stride, int valid) {
  return valid == kTileP && (row_stride & 1) == 0 && (reinterpret_cast<uintptr_t>(base) & 15) == 0;
}

// R2C split (in place in shared memory, rows 0..M). Bins 1..M-1 are scaled by
// `interior`. In the swizzled tile the pencils p, p+1 (p even) of a row share
// one 16-byte chunk, so a thread takes the pair (k, M-k) of two pencils.
template <int M, int THREADS>
__device__ __forceinline__ void r2c_post(float2* sm, const float2* tw2, float interior) {
  constexpr int NPAIR = M / 2 + 1;
  for (int it = threadIdx.x; it < NPAIR * 8; it += THREADS) {
    const int p = (it & 7) << 1, k = it >> 3;
    float4* rk = reinterpret_cast<float4*>(sm + swz(k, p));
    if (k == 0) {
      const float4 z0 = *rk;
      *rk = make_float4(z0.x + z0.y, 0.f, z0.z + z0.w, 0.f);
      *reinterpret_cast<float4*>(sm + swz(M, p)) = make_float4(z0.x - z0.y, 0.f, z0.z - z0.w, 0.f);
    } else if (2 * k < M) {
      float4* rm = reinterpret_cast<float4*>(sm + swz(M - k, p));
      const float4 A = *rk, B = *rm;
      const float2 w = tw2[k];
      float2 xk0, xm0, xk1, xm1;
      r2c_split_pair(lo2(A), lo2(B), w, xk0, xm0);
      r2c_split_pair(hi2(A), hi2(B), w, xk1, xm1);
      *rk = cat2(cscale(xk0, interior), cscale(xk1, interior));
      *rm = cat2(cscale(xm0, interior), cscale(xm1, interior));
    } else if (2 * k == M) {
      const float4 A = *rk;
      *rk = cat2(cscale(cconj(lo2(A)), interior), cscale(cconj(hi2(A)), interior));
    }
  }
  __syncthreads();
}

// The R2C split fused with the column-side store of rows 0..M: the pair
// (k, M-k) is split from the transform in shared memory and both bins go
// straight to global memory, with the roundings of r2c_post then col_store
// but without the shared-memory write-back and its barrier. Full, aligned
// tiles move two pencils per 16-byte access (8 lanes per 128-byte line).
// UNIT: interior = scale = 1 (the forward transform), no multiplies.
template <int M, int THREADS, bool UNIT>
__device__ __forceinline__ void r2c_post_col_store_impl(const float2* sm, const float2* tw2, float interior,
                                                        const TileIO& io) {
  constexpr int NPAIR = M / 2 + 1;
  const float sc = io.scale;
  auto fin = [&](float2 x) { return UNIT ? x : cscale(cscale(x, interior), sc); };
  if (pair_vec_ok(io.gout, io.out_n, io.valid)) {
    for (int it = threadIdx.x; it < NPAIR * 8; it += THREADS) {
      const int p = (it & 7) << 1, k = it >> 3;
      float4* g = reinterpret_cast<float4*>(io.gout + p);
      const long long rk = (long long)k * (io.out_n >> 1), rm = (long long)(M - k) * (io.out_n >> 1);
      const float4 A = *reinterpret_cast<const float4*>(sm + swz(k, p));
      if (k == 0) {
        if (UNIT) {
          st_data4(g, make_float4(A.x + A.y, 0.f, A.z + A.w, 0.f));
          st_data4(g + rm, make_float4(A.x - A.y, 0.f, A.z - A.w, 0.f));
        } else {
          st_data4(g, make_float4((A.x + A.y) * sc, 0.f * sc, (A.z + A.w) * sc, 0.f * sc));
          st_data4(g + rm, make_float4((A.x - A.y) * sc, 0.f * sc, (A.z - A.w) * sc, 0.f * sc));
        }
      } else if (2 * k < M) {
        const float4 B = *reinterpret_cast<const float4*>(sm + swz(M - k, p));
        const float2 w = tw2[k];
        float2 xk0, xm0, xk1, xm1;
        r2c_split_pair(lo2(A), lo2(B), w, xk0, xm0);
        r2c_split_pair(hi2(A), hi2(B), w, xk1, xm1);
        st_data4(g + rk, cat2(fin(xk0), fin(xk1)));
        st_data4(g + rm, cat2(fin(xm0), fin(xm1)));
      } else if (2 * k == M) {
        st_data4(g + rk, cat2(fin(cconj(lo2(A))), fin(cconj(hi2(A)))));
      }
    }
    return;
  }
  for (int it = threadIdx.x; it < NPAIR * 16; it += THREADS) {
    const int p = it & 15, k = it >> 4;
    if (p >= io.valid) continue;
    float2* g = io.gout + p;
    if (k == 0) {
      const float2 z0 = sm[swz(0, p)];
      if (UNIT) {
        st_data(g, make_float2(z0.x + z0.y, 0.f));
        st_data(g + M * io.out_n, make_float2(z0.x - z0.y, 0.f));
      } else {
        st_data(g, make_float2((z0.x + z0.y) * sc, 0.f * sc));
        st_data(g + M * io.out_n, make_float2((z0.x - z0.y) * sc, 0.f * sc));
      }
    } else if (2 * k < M) {
      float2 xk, xm;
      r2c_split_pair(sm[swz(k, p)], sm[swz(M - k, p)], tw2[k], xk, xm);
      st_data(g + k * io.out_n, fin(xk));
      st_data(g + (M - k) * io.out_n, fin(xm));
    } else if (2 * k == M) {
      st_data(g + k * io.out_n, fin(cconj(sm[swz(k, p)])));
    }
  }
}

template <int M, int THREADS>
__device__ __forceinline__ void r2c_post_col_store(const float2* sm, const float2* tw2, float interior,
                                                   const TileIO& io) {
  if (interior == 1.f && io.scale == 1.f) r2c_post_col_store_impl<M, THREADS, true>(sm, tw2, interior, io);
  else r2c_post_col_store_impl<M, THREADS, false>(sm, tw2, interior, io);
}

// C2R merge (in place, reads rows 0..M, writes rows 0..M-1). Only the real
// parts of X[0] and X[M] enter (the Hermitian projection); the inverse
// length-M FFT of Z then gives x[2m] + i x[2m+1]. Pencil pairs as in r2c_post.
template <int M, int THREADS>
__device__ __forceinline__ void c2r_pre(float2* sm, const float2* tw2, float interior) {
  constexpr int NPAIR = M / 2 + 1;
  for (int it = threadIdx.x; it < NPAIR * 8; it += THREADS) {
    const int p = (it & 7) << 1, k = it >> 3;
    float4* rk = reinterpret_cast<float4*>(sm + swz(k, p));
    if (k == 0) {
      const float4 a = *rk, c = *reinterpret_cast<const float4*>(sm + swz(M, p));
      *rk = make_float4(a.x + c.x, a.x - c.x, a.z + c.z, a.z - c.z);
    } else if (2 * k < M) {
      float4* rm = reinterpret_cast<float4*>(sm + swz(M - k, p));
      const float4 A = *rk, B = *rm;
      const float2 w = tw2[k];
      float2 zk0, zm0, zk1, zm1;
      c2r_merge_pair(cscale(lo2(A), interior), cscale(lo2(B), interior), w, zk0, zm0);
      c2r_merge_pair(cscale(hi2(A), interior), cscale(hi2(B), interior), w, zk1, zm1);
      *rk = cat2(zk0, zk1);
      *rm = cat2(zm0, zm1);
    } else if (2 * k == M) {
      const float2 x0 = cscale(lo2(*rk), interior), x1 = cscale(hi2(*rk), interior);
      *rk = make_float4(2.f * x0.x, -2.f * x0.y, 2.f * x1.x, -2.f * x1.y);
    }
  }
  __syncthreads();
}

// The fused C2R column load for full, aligned tiles (pair_vec_ok), split so
// that a tile loop can issue part of a tile's loads early: the first kEarly
// of the thread's pairs (k, M-k) of two pencils are read into A, B ahead of
// time, the rest when the tile is merged into rows k and M-k.
template <int M, int THREADS>
struct C2REarlyLoads {
  static constexpr int kIters = ((M / 2 + 1) * 8 + THREADS - 1) / THREADS;
  static constexpr int kEarly = 1;
  float4 A[kEarly], B[kEarly];
};

template <int M>
__device__ __forceinline__ void c2r_load_pair(const TileIO& io, int it, float4& a, float4& b) {
  const int p = (it & 7) << 1, k = it >> 3;
  const float4* g = reinterpret_cast<const float4*>(io.gin + p);
  a = ld_data4(g + (long long)k * (io.in_n >> 1));
  b = ld_data4(g + (long long)(M - k) * (io.in_n >> 1));  // k = 0: row M; 2k = M: row k again
}

// UNIT: interior = 1 (the inverse transform), no multiplies.
template <int M, bool UNIT = false>
__device__ __forceinline__ void c2r_merge_pair_to(float2* sm, const float2* tw2, float interior, int it, float4 a,
                                                  float4 c) {
  const int p = (it & 7) << 1, k = it >> 3;
  float4* sk = reinterpret_cast<float4*>(sm + swz(k, p));
  if (k == 0) {
    *sk = make_float4(a.x + c.x, a.x - c.x, a.z + c.z, a.z - c.z);
  } else if (2 * k < M) {
    const float2 w = tw2[k];
    float2 zk0, zm0, zk1, zm1;
    if (UNIT) {
      c2r_merge_pair(lo2(a), lo2(c), w, zk0, zm0);
      c2r_merge_pair(hi2(a), hi2(c), w, zk1, zm1);
    } else {
      c2r_merge_pair(cscale(lo2(a), interior), cscale(lo2(c), interior), w, zk0, zm0);
      c2r_merge_pair(cscale(hi2(a), interior), cscale(hi2(c), interior), w, zk1, zm1);
    }
    *sk = cat2(zk0, zk1);
    *reinterpret_cast<float4*>(sm + swz(M - k, p)) = cat2(zm0, zm1);
  } else if (2 * k == M) {
    const float2 x0 = UNIT ? lo2(a) : cscale(lo2(a), interior), x1 = UNIT ? hi2(a) : cscale(hi2(a), interior);
    *sk = make_float4(2.f * x0.x, -2.f * x0.y, 2.f * x1.x, -2.f * x1.y);
  }
}

template <int M, int THREADS>
__device__ __forceinline__ void c2r_issue_early(const TileIO& io, C2REarlyLoads<M, THREADS>& r) {
  static_for<C2REarlyLoads<M, THREADS>::kEarly>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    const int it = threadIdx.x + i * THREADS;
    if (it < (M / 2 + 1) * 8) c2r_load_pair<M>(io, it, r.A[i], r.B[i]);
  });
}

// Merge a tile whose early loads are in r; ends with the barrier before the first pass.
template <int M, int THREADS>
__device__ __forceinline__ void c2r_merge_rest(float2* sm, const float2* tw2, float interior, const TileIO& io,
                                               const C2REarlyLoads<M, THREADS>& r) {
  using E = C2REarlyLoads<M, THREADS>;
  constexpr int NPAIR = M / 2 + 1;
  static_for<E::kIters - E::kEarly>([&](auto ic) {
    constexpr int i = decltype(ic)::value + E::kEarly;
    const int it = threadIdx.x + i * THREADS;
    if (it < NPAIR * 8) {
      float4 a, c;
      c2r_load_pair<M>(io, it, a, c);
      c2r_merge_pair_to<M>(sm, tw2, interior, it, a, c);
    }
  });
  static_for<E::kEarly>([&](auto ic) {
    constexpr int i = decltype(ic)::value;
    const int it = threadIdx.x + i * THREADS;
    if (it < NPAIR * 8) c2r_merge_pair_to<M>(sm, tw2, interior, it, r.A[i], r.B[i]);
  });
  __syncthreads();
}

// The column-side load of bins 0..M fused with the C2R merge: the pair
// (k, M-k) is read from global memory and merged into rows k and M-k of the
// tile, with the arithmetic of c2r_pre. Full, aligned tiles read two pencils
// per 16-byte access. Ends with the barrier that orders the tile before the
// first pass.
template <int M, int THREADS>
__device__ __forceinline__ void col_load_c2r_pre(float2* sm, const float2* tw2, float interior, const TileIO& io) {
  constexpr int NPAIR = M / 2 + 1;
  if (pair_vec_ok(io.gin, io.in_n, io.valid)) {
    // the loads of CH consecutive pairs of the thread are issued before their
    // merges, so the thread waits for one global-memory latency per CH pairs
    constexpr int ITERS = (NPAIR * 8 + THREADS - 1) / THREADS;
    constexpr int CH = 1;
    static_for<(ITERS + CH - 1) / CH>([&](auto cc) {
      constexpr int c0 = decltype(cc)::value * CH;
      float4 A[CH], B[CH];
      static_for<CH>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const int it = threadIdx.x + (c0 + i) * THREADS;
        if (c0 + i < ITERS && it < NPAIR * 8) {
          const int p = (it & 7) << 1, k = it >> 3;
          const float4* g = reinterpret_cast<const float4*>(io.gin + p);
          A[i] = ld_data4(g + (long long)k * (io.in_n >> 1));
          B[i] = ld_data4(g + (long long)(M - k) * (io.in_n >> 1));  // k = 0: row M; 2k = M: row k again
        }
      });
      static_for<CH>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const int it = threadIdx.x + (c0 + i) * THREADS;
        if (c0 + i < ITERS && it < NPAIR * 8) {
          const int p = (it & 7) << 1, k = it >> 3;
          float4* sk = reinterpret_cast<float4*>(sm + swz(k, p));
          const float4 a = A[i], c = B[i];
          if (k == 0) {
            *sk = make_float4(a.x + c.x, a.x - c.x, a.z + c.z, a.z - c.z);
          } else if (2 * k < M) {
            const float2 w = tw2[k];
            float2 zk0, zm0, zk1, zm1;
            c2r_merge_pair(cscale(lo2(a), interior), cscale(lo2(c), interior), w, zk0, zm0);
            c2r_merge_pair(cscale(hi2(a), interior), cscale(hi2(c), interior), w, zk1, zm1);
            *sk = cat2(zk0, zk1);
            *reinterpret_cast<float4*>(sm + swz(M - k, p)) = cat2(zm0, zm1);
          } else if (2 * k == M) {
            const float2 x0 = cscale(lo2(a), interior), x1 = cscale(hi2(a), interior);
            *sk = make_float4(2.f * x0.x, -2.f * x0.y, 2.f * x1.x, -2.f * x1.y);
          }
        }
      });
    });
    __syncthreads();
    return;
  }
  for (int it = threadIdx.x; it < NPAIR * 16; it += THREADS) {
    const int p = it & 15, k = it >> 4;
    const bool ok = p < io.valid;
    const float2* g = io.gin + p;
    const float2 z = make_float2(0.f, 0.f);
    if (k == 0) {
      const float a = ok ? ld_data(g).x : 0.f, c = ok ? ld_data(g + M * io.in_n).x : 0.f;
      sm[swz(0, p)] = make_float2(a + c, a - c);
    } else if (2 * k < M) {
      const float2 xk = cscale(ok ? ld_data(g + k * io.in_n) : z, interior);
      const float2 xm = cscale(ok ? ld_data(g + (M - k) * io.in_n) : z, interior);
      c2r_merge_pair(xk, xm, tw2[k], sm[swz(k, p)], sm[swz(M - k, p)]);
    } else if (2 * k == M) {
      const float2 xk = cscale(ok ? ld_data(g + k * io.in_n) : z, interior);
      sm[swz(k, p)] = make_float2(2.f * xk.x, -2.f * xk.y);
    }
  }
  __syncthreads();
}

// Poisson multiplier -1/|k|^2 (k = 0 -> 0) on the z pencils of the R2C half
// spectrum, folded with the 1/N of the inverse. Pencil p has kx = gfirst + p,
// the tile's outer index is ky, row n is kz.
template <int L, int THREADS>
__device__ __forceinline__ void poisson_multiply(float2* sm, int gfirst, int ky_idx, int ny, float inv_n) {
  const float ky = (float)(ky_idx <= ny / 2 ? ky_idx : ky_idx - ny);
  for (int it = threadIdx.x; it < L * 16; it += THREADS) {
    const int p = it & 15, n = it >> 4;
    const float kx = (float)(gfirst + p);
    const float kz = (float)(n <= L / 2 ? n : n - L);
    const float k2 = kx * kx + ky * ky + kz * kz;
    const float m = k2 > 0.f ? -inv_n / k2 : 0.f;
    float2 v = sm[swz(n, p)];
    sm[swz(n, p)] = make_float2(v.x * m, v.y * m);
  }
  __syncthreads();
}

// ------------------------------------------ bounded z: DCT-II / DCT-III by FFT
//
// Along a bounded axis with Neumann walls (cell centres z_n = (n + 1/2) dz)
// the Poisson solve expands in cosines: DCT-II (FFTW's REDFT10)
//   Y_k = 2 sum_n x_n cos(pi k (2n + 1) / 2L),
// and back with DCT-III (REDFT01) x_n = Y_0 + 2 sum_{k>0} Y_k cos(pi k (2n + 1) / 2L),
// which returns 2L x. Both run as one length-L complex FFT each (the
// reordering v_m = x_2m, v_(L-1-m) = x_(2m+1) of Makhoul's method): with
// V = FFT(v) and V_c[k] = conj V[(L - k) mod L], the real and imaginary parts
// of x transform separately, Vr = (V + V_c) / 2, Vi = (V - V_c) / 2i, and
//   Y_k = 2 Re(W_k Vr_k) + 2 i Re(W_k Vi_k),  W_k = exp(-i pi k / 2L);
// backwards V'_k = conj(W_k) (Yr_k - i Yr_(L-k)) + i conj(W_k) (Yi_k - i Yi_(L-k))
// (Y_L = 0) and the unscaled inverse FFT of V' is v.

// position of element i of a pencil in the reordered sequence v
__device__ __forceinline__ int dct_pos(int i, int L) { return (i & 1) ? L - 1 - (i >> 1) : (i >> 1); }

// Pair (k, j = L - k) of the DCT-II post-processing: from V_k = A, V_j = B
// (the FFT of the reordered pencil) to Y_k, Y_j.
__device__ __forceinline__ void dct2_post_pair(float2 A, float2 B, float2 Wk, float2 Wj, float2& Yk, float2& Yj) {
  auto one = [](float2 a, float2 b, float2 w) {
    // Vr = (a + conj b) / 2, Vi = (a - conj b) / 2i; Y = 2 Re(w Vr) + 2 i Re(w Vi)
    const float2 vr = make_float2(0.5f * (a.x + b.x), 0.5f * (a.y - b.y));
    const float2 vi = make_float2(0.5f * (a.y + b.y), -0.5f * (a.x - b.x));
    return make_float2(2.f * (w.x * vr.x - w.y * vr.y), 2.f * (w.x * vi.x - w.y * vi.y));
  };
  Yk = one(A, B, Wk);
  Yj = one(B, A, Wj);
}

// Pair (k, j = L - k), k >= 1, of the DCT-III pre-processing:
// V'_k = conj(W_k) (Yr_k - i Yr_j) + i conj(W_k) (Yi_k - i Yi_j) = conj(W_k) (Yr_k + Yi_j + i (Yi_k - Yr_j)).
__device__ __forceinline__ void dct3_pre_pair(float2 Yk, float2 Yj, float2 Wk, float2 Wj, float2& Vk, float2& Vj) {
  Vk = cmul(cconj(Wk), make_float2(Yk.x + Yj.y, Yk.y - Yj.x));
  Vj = cmul(cconj(Wj), make_float2(Yj.x + Yk.y, Yj.y - Yk.x));
}

// DCT-II of every pencil's FFT (rows 0..L-1), multiply by the bounded Poisson
// symbol, and prepare the DCT-III FFT input, pair (k, L - k) per item. The
// symbol is -inv_n / (kx^2 + ky^2 + kz^2) with kz = k (cosine index), kx the
// pencil's half-spectrum bin, ky the outer index folded to [-ny/2, ny/2].
template <int L, int THREADS>
__device__ __forceinline__ void dct_poisson_bounded(float2* sm, const float2* w4, int gfirst, int ky_idx, int ny,
                                                    float inv_n) {
  constexpr int NPAIR = L / 2 + 1;
  const float ky = (float)(ky_idx <= ny / 2 ? ky_idx : ky_idx - ny);
  for (int it = threadIdx.x; it < NPAIR * 16; it += THREADS) {
    const int p = it & 15, k = it >> 4;
    const int j = k == 0 ? 0 : L - k;
    if (k > j) continue;  // the pair was taken by item (j, k)
    const float kx = (float)(gfirst + p);
    float2 Yk, Yj;
    dct2_post_pair(sm[swz(k, p)], sm[swz(j, p)], w4[k], w4[j], Yk, Yj);
    const float kz_k = (float)k, kz_j = (float)j;
    const float k2k = kx * kx + ky * ky + kz_k * kz_k, k2j = kx * kx + ky * ky + kz_j * kz_j;
    Yk = cscale(Yk, k2k > 0.f ? -inv_n / k2k : 0.f);
    Yj = cscale(Yj, k2j > 0.f ? -inv_n / k2j : 0.f);
    if (k == 0) {
      sm[swz(0, p)] = Yk;  // Y_L = 0 and W_0 = 1: V'_0 = Y_0
    } else {
      float2 Vk, Vj;
      dct3_pre_pair(Yk, Yj, w4[k], w4[j], Vk, Vj);
      sm[swz(k, p)] = Vk;
      if (j != k) sm[swz(j, p)] = Vj;
    }
  }
  __syncthreads();
}

// DCT-II post-processing alone (rows 0..L-1 become Y_0..Y_(L-1)), in place.
template <int L, int THREADS>
__device__ __forceinline__ void dct2_post(float2* sm, const float2* w4) {
  constexpr int NPAIR = L / 2 + 1;
  for (int it = threadIdx.x; it < NPAIR * 16; it += THREADS) {
    const int p = it & 15, k = it >> 4;
    const int j = k == 0 ? 0 : L - k;
    if (k > j) continue;
    float2 Yk, Yj;
    dct2_post_pair(sm[swz(k, p)], sm[swz(j, p)], w4[k], w4[j], Yk, Yj);
    sm[swz(k, p)] = Yk;
    if (j != k) sm[swz(j, p)] = Yj;
  }
  __syncthreads();
}

// DCT-III pre-processing alone (rows 0..L-1 hold Y, become the FFT input V'), in place.
template <int L, int THREADS>
__device__ __forceinline__ void dct3_pre(float2* sm, const float2* w4) {
  constexpr int NPAIR = L / 2 + 1;
  for (int it = threadIdx.x; it < NPAIR * 16; it += THREADS) {
    const int p = it & 15, k = it >> 4;
    const int j = k == 0 ? 0 : L - k;
    if (k > j || k == 0) continue;  // V'_0 = Y_0 stays
    float2 Vk, Vj;
    dct3_pre_pair(sm[swz(k, p)], sm[swz(j, p)], w4[k], w4[j], Vk, Vj);
    sm[swz(k, p)] = Vk;
    if (j != k) sm[swz(j, p)] = Vj;
  }
  __syncthreads();
}

// ------------------------------------------------------------- tile driver

template <int L, int DIR, int KIND>
struct TileShape {
  static constexpr int kThreads = threads_for(L);
  static constexpr int kRows = L + 1;  // one spare row for the Nyquist bin of R2C/C2R
  static constexpr int kSmemTile = kRows * kTileP;  // float2 elements
};

__device__ __forceinline__ TileIO make_io(const StageDesc& d, long long tile, int& o_out, int& g0_out) {
  TileIO io;
  // 32-bit decode (tile counts stay below 2^32): 64-bit division is a subroutine call
  const unsigned t32 = (unsigned)tile;
  const unsigned gc = t32 % (unsigned)d.n_gchunks;
  const unsigned rest = t32 / (unsigned)d.n_gchunks;
  const int o = (int)(rest % (unsigned)d.n_outer);
  const int b = (int)(rest / (unsigned)d.n_outer);
  const int g0 = (int)gc * kTileP;
  io.valid = min(kTileP, d.n_group - g0);
  io.gin = d.in + b * d.in_b + o * d.in_o + g0 * d.in_g;
  io.gout = d.out + b * d.out_b + o * d.out_o + g0 * d.out_g;
  io.in_g = d.in_g;
  io.in_n = d.in_n;
  io.out_g = d.out_g;
  io.out_n = d.out_n;
  io.scale = d.scale;
  o_out = o;
  g0_out = g0;
  return io;
}

// Process one tile of one stage. THREADS may exceed threads_for(L) (the
// persistent kernel runs several lengths with one block size); the extra
// groups then share the butterflies.
// idle: the team runs the tile's barriers and arithmetic but reads and writes
// nothing in global memory (a batched ticket whose last teams have no tile).
template <int L, int DIR, int KIND, int THREADS, int PREC = kPrecFP32>
__device__ __forceinline__ void process_tile(const StageDesc& d, long long tile, float2* sm, const float2* tw,
                                             const float2* tw2, bool idle = false) {
  int o, g0;
  TileIO io = make_io(d, tile, o, g0);
  if (idle) io.valid = 0;
  const bool row_in = d.in_mode == kRow, row_out = d.out_mode == kRow;
  const bool inplace = d.in == d.out;

  if constexpr (KIND == kIdentity) {
    // pure redistribution: unpack into the tile, pack out of it
    if (row_in) row_load<THREADS, L>(sm, io);
    else col_load<THREADS, L>(sm, io);
    __syncthreads();
    if (row_out) row_store<THREADS, L>(sm, io);
    else col_store<THREADS, L>(sm, io);
  } else if constexpr (KIND == kPlain) {
    if (row_in) {
      row_load<THREADS, L>(sm, io);
      __syncthreads();
      if (row_out) {
        fft_passes<L, DIR, THREADS, false, false, false, 0, 0, PREC>(sm, tw, io);
        row_store<THREADS, L>(sm, io);
      } else {
        fft_passes<L, DIR, THREADS, false, true, false, 0, 0, PREC>(sm, tw, io);
      }
    } else {
      if (row_out) {
        fft_passes<L, DIR, THREADS, true, false, false, 0, 0, PREC>(sm, tw, io);
        row_store<THREADS, L>(sm, io);
      } else if (inplace) {
        fft_passes<L, DIR, THREADS, true, true, true, 0, 0, PREC>(sm, tw, io);
      } else {
        fft_passes<L, DIR, THREADS, true, true, false, 0, 0, PREC>(sm, tw, io);
      }
    }
  } else if constexpr (KIND == kR2CPost) {
    // real rows viewed as L complex pairs -> L+1 half-spectrum bins
    row_load<THREADS, L>(sm, io);
    __syncthreads();
    fft_passes<L, -1, THREADS, false, false, false>(sm, tw, io);
    if (row_out) {
      r2c_post<L, THREADS>(sm, tw2, d.interior);
      row_store<THREADS, L + 1>(sm, io);
    } else {
      r2c_post_col_store<L, THREADS>(sm, tw2, d.interior, io);
    }
  } else if constexpr (KIND == kC2RPre) {
    // L+1 half-spectrum bins -> L complex pairs of real output
    if (row_in) {
      row_load<THREADS, L + 1>(sm, io);
      __syncthreads();
      c2r_pre<L, THREADS>(sm, tw2, d.interior);
    } else {
      col_load_c2r_pre<L, THREADS>(sm, tw2, d.interior, io);
    }
    fft_passes<L, +1, THREADS, false, false, false>(sm, tw, io);
    row_store<THREADS, L>(sm, io);
  } else if constexpr (KIND == kPoissonZB) {
    // bounded z pencils: reorder into v, FFT, DCT-II + multiply + DCT-III input, FFT, reorder back
    TileIO io_nos = io;
    io_nos.scale = 1.f;
    for (int it = threadIdx.x; it < L * 16; it += THREADS) {
      int p, n;
      if (row_in) {  // lanes along the row
        n = it % L;
        p = it / L;
      } else {  // lanes along the pencils
        p = it & 15;
        n = it >> 4;
      }
      const float2 a = (p < io.valid) ? ld_data(io.gin + p * io.in_g + n * io.in_n) : make_float2(0.f, 0.f);
      sm[swz(dct_pos(n, L), p)] = a;
    }
    __syncthreads();
    fft_passes<L, -1, THREADS, false, false, false>(sm, tw, io_nos);
    dct_poisson_bounded<L, THREADS>(sm, tw2, g0, o, d.pz_ny, d.scale);
    fft_passes<L, +1, THREADS, false, false, false>(sm, tw, io_nos);
    for (int it = threadIdx.x; it < L * 16; it += THREADS) {
      int p, n;
      if (row_out) {
        n = it % L;
        p = it / L;
      } else {
        p = it & 15;
        n = it >> 4;
      }
      if (p < io.valid) st_data(io.gout + p * io.out_g + n * io.out_n, sm[swz(dct_pos(n, L), p)]);
    }
  } else if constexpr (KIND == kDct2 || KIND == kDst2 || KIND == kDct3 || KIND == kDst3) {
    // real-to-real along the stage's axis (linear, so complex pencils transform their real and imaginary
    // parts alike). DST-II(x)_k = DCT-II(s x)_(L-1-k) and DST-III(Y)_n = s_n DCT-III(reversed Y)_n,
    // s_n = (-1)^n: the sine kinds flip signs and reverse order on the way in or out.
    constexpr bool kFwd = KIND == kDct2 || KIND == kDst2;
    constexpr bool kSine = KIND == kDst2 || KIND == kDst3;
    TileIO io_nos = io;
    io_nos.scale = 1.f;
    for (int it = threadIdx.x; it < L * 16; it += THREADS) {
      int p, n;
      if (row_in) {
        n = it % L;
        p = it / L;
      } else {
        p = it & 15;
        n = it >> 4;
      }
      float2 a = (p < io.valid) ? ld_data(io.gin + p * io.in_g + n * io.in_n) : make_float2(0.f, 0.f);
      int row;
      if constexpr (kFwd) {
        row = dct_pos(n, L);
        if (kSine && (n & 1)) a = make_float2(-a.x, -a.y);
      } else {
        row = kSine ? L - 1 - n : n;
      }
      sm[swz(row, p)] = a;
    }
    __syncthreads();
    if constexpr (kFwd) {
      fft_passes<L, -1, THREADS, false, false, false>(sm, tw, io_nos);
      dct2_post<L, THREADS>(sm, tw2);
    } else {
      dct3_pre<L, THREADS>(sm, tw2);
      fft_passes<L, +1, THREADS, false, false, false>(sm, tw, io_nos);
    }
    const float sc = io.scale;
    for (int it = threadIdx.x; it < L * 16; it += THREADS) {
      int p, n;
      if (row_out) {
        n = it % L;
        p = it / L;
      } else {
        p = it & 15;
        n = it >> 4;
      }
      if (p < io.valid) {
        float2 v;
        if constexpr (kFwd) {
          v = sm[swz(kSine ? L - 1 - n : n, p)];
        } else {
          v = sm[swz(dct_pos(n, L), p)];
          if (kSine && (n & 1)) v = make_float2(-v.x, -v.y);
        }
        st_data(io.gout + p * io.out_g + n * io.out_n, cscale(v, sc));
      }
    }
  } else if constexpr (KIND == kPoissonZ) {
    // z pencils of the half spectrum: forward, multiply, inverse, in one tile
    TileIO io_nos = io;
    io_nos.scale = 1.f;
    if (row_in) {
      row_load<THREADS, L>(sm, io);
      __syncthreads();
      fft_passes<L, -1, THREADS, false, false, false>(sm, tw, io_nos);
    } else {
      fft_passes<L, -1, THREADS, true, false, false>(sm, tw, io_nos);
    }
    poisson_multiply<L, THREADS>(sm, g0, o, d.pz_ny, d.scale);
    if (row_out) {
      fft_passes<L, +1, THREADS, false, false, false>(sm, tw, io_nos);
      row_store<THREADS, L>(sm, io_nos);
    } else {
      fft_passes<L, +1, THREADS, false, true, false>(sm, tw, io_nos);
    }
  }
}

// Copy a stage's twiddle tables into shared memory.
template <int L, int THREADS>
__device__ __forceinline__ void load_twiddles(float2* tw_s, float2* tw2_s, const StageDesc& d, bool need_tw2) {
  constexpr int TWL = tw_table_len(L);
  for (int i = threadIdx.x; i < TWL; i += THREADS) tw_s[i] = d.tw[i];
  if (need_tw2)
    for (int i = threadIdx.x; i <= L; i += THREADS) tw2_s[i] = d.tw2[i];
}

}  // namespace gbfft
