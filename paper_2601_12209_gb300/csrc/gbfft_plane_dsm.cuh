// Slab in-plane stage pair of a real transform with each plane's intermediate
// kept in distributed shared memory.
//
// Section III-A's slab variant transforms each z-plane in 2D, then does one
// transpose and the 1D transforms along z: two passes over the array in HBM,
// where the pencil variant takes three. On one GPU the 2D transform of a
// plane is the x stage and the y stage. Their intermediate, an R2C plane of
// 512-point rows (257 x ny complex, 1.05 MB at ny = 512), fits in the shared
// memory of an 8-CTA cluster, so it never leaves the chip.
//
// Columns. Spectrum columns kx = 1..255 belong to CTA kx / 32 (its column
// kx % 32). Bins 0 and 256 of a real row's half spectrum are real, so the
// columns kx = 0 and kx = 256 travel packed as one complex column
// a + i b = X[y][0] + i X[y][256], column 0 of CTA 0: every CTA owns 32
// columns of ny values. The y transform of the packed column,
// Z = FFT_y(a + i b), separates into A[k] = (Z[k] + conj Z[-k]) / 2 and
// B[k] = (Z[k] - conj Z[-k]) / 2i. The inverse packs the Hermitian parts
// Ah[k] = (A[k] + conj A[-k]) / 2 and Bh of its two real-bin columns as
// Ah + i Bh: the inverse y transform of that column is Re IFFT(A) + i Re IFFT(B),
// exactly the real parts of bins 0 and 256 that the C2R merge reads.
//
// Forward, per plane:
//   (A) CTA r transforms rows 64 r .. 64 r + 63 (one warp per row: the
//       warp-per-pencil length-256 body, then the R2C split in the warp's
//       region) and stores each bin into the column buffer of the CTA that
//       owns its column, two rows per 16-byte st.shared::cluster;
//   a cluster barrier (release / acquire) makes the stores visible;
//   (B) warp j transforms column j along y in place (the column's storage
//       doubles as the warp's transpose buffer), and the CTA writes its 32
//       columns of every row ky to HBM;
//   a second cluster barrier frees the buffers for the next plane.
// Inverse, per plane:
//   (A) CTA r loads its 32 columns of the plane's spectrum from HBM and
//       transforms them along y in place;
//   a cluster barrier;
//   (B) each CTA gathers the 257 bins of its rows from the 8 column buffers
//       (16-byte ld.shared::cluster), merges them (C2R) and transforms them
//       along x in the warps' regions, and writes the real rows;
//   a cluster barrier.
// Each plane crosses HBM once in and once out. There are no spin waits:
// every CTA of a cluster runs the same planes and meets the same barriers.
#pragma once
#include "gbfft_plane.cuh"
#include "gbfft_warp_tile.cuh"

namespace gbfft {

struct PlaneDsmKernel {
  int ny, dir;
  const void* fn;
  int threads;
  size_t smem;
};

std::vector<PlaneDsmKernel>& plane_dsm_registry();

constexpr int kDsmCta = 8;                  // CTAs per plane cluster
constexpr int kDsmM = 256;                  // complex length of the x stage (512-point real rows)
constexpr int kDsmCols = kDsmM / kDsmCta;   // packed spectrum columns per CTA
constexpr int kDsmWarps = 32;               // one warp per column (y) or per row of a row tile (x)
constexpr int kDsmThreads = 32 * kDsmWarps;

template <int NY>
struct DsmGeom {
  static constexpr int kRows = NY / kDsmCta;           // x-stage rows of one CTA
  static constexpr int kRowTiles = kRows / kDsmWarps;  // row tiles of 32 rows
  static constexpr int kNeed = NY > WarpGeom<NY>::kBuf ? NY : WarpGeom<NY>::kBuf;
  // column pitch: a column and its warp's transpose buffer; = 2 mod 16, so
  // every column starts on 16 bytes (the 16-byte cluster accesses) and the
  // row-wise reads of the output pass spread over all banks
  static constexpr int kColPitch = kNeed + ((18 - kNeed % 16) % 16);
  static constexpr int kRegionX = WarpGeom<kDsmM>::kRegion;  // x-stage region of a warp (odd by 16)
  static_assert(kColPitch % 16 == 2 && kColPitch >= kNeed, "column pitch");
  static_assert(kRows % kDsmWarps == 0 && kRowTiles >= 1, "whole row tiles");
  static_assert(kDsmWarps * kRegionX >= NY, "the regions hold the separated bin-256 column");
  static_assert(kDsmWarps == kDsmCols && (NY * kDsmCols) % kDsmThreads == 0 && (kDsmM * 16) % kDsmThreads == 0,
                "one warp per column; whole passes of the block over a plane's columns and a tile's bins");
};

template <int NY>
constexpr size_t plane_dsm_smem_bytes() {
  using G = DsmGeom<NY>;
  // column buffer, x regions, x twiddles [k1][t] + W_32 + W_512^k (k <= 256), y twiddles + W_32
  return sizeof(float2) * ((size_t)kDsmCols * G::kColPitch + (size_t)kDsmWarps * G::kRegionX + kDsmM + 32 +
                           (kDsmM + 1) + NY + 32);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// the shared::cluster address of shared::cta address a in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_map(uint32_t a, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ __forceinline__ void st_cluster4(uint32_t a, float4 v) {
  asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
               : "memory");
}

__device__ __forceinline__ float4 ld_cluster4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a)
               : "memory");
  return v;
}

// Length-NY transform of column j (warp j) in place: natural order in, natural
// order out, times `scale`. The column's storage is the transpose buffer.
template <int NY, int DIR>
__device__ __forceinline__ void dsm_column_fft(float2* cw, const float2* twy, const float2* w32y, float scale) {
  using G = WarpGeom<NY>;
  constexpr int R1 = G::R1, C = G::C;
  const int lane = threadIdx.x & 31;
  const int k1 = lane / C, c = lane % C;
  const int m = C == 2 ? c : ((c >> 1) + 2 * (c & 1));
  float2 v[R1];
#pragma unroll
  for (int i = 0; i < R1; ++i) v[i] = cw[lane + 32 * i];
  __syncwarp();
  warp_steps12<NY, DIR>(v, cw, twy, w32y, lane);
  __syncwarp();
  warp_steps345<NY, DIR>(v, cw, w32y);
  __syncwarp();
#pragma unroll
  for (int k = 0; k < R1; ++k) cw[k1 + R1 * k + R1 * R1 * m] = cscale(v[k], scale);
  __syncwarp();
}

// Cluster c of the grid takes planes c, c + clusters, ... (plane = batch entry
// x outer index of both stages). s1 / s2: the pair's descriptors in pipeline
// order (forward: R2C x stage, then y; inverse: y, then C2R x stage). The
// x stage's rows are contiguous (in_n / out_n = 1); the y stage's side in HBM
// is the natural spectrum (kx stride 1, ky stride nxc).
template <int NY, int DIR>
__global__ void __launch_bounds__(kDsmThreads, 1) plane_dsm_kernel(StageDesc s1, StageDesc s2) {
  using G = DsmGeom<NY>;
  constexpr int CP = G::kColPitch, RX = G::kRegionX, M = kDsmM;
  constexpr int R1X = WarpGeom<M>::R1, CX = WarpGeom<M>::C;
  extern __shared__ float4 smem4[];
  float2* col = reinterpret_cast<float2*>(smem4);  // [kDsmCols][CP]
  float2* xr = col + kDsmCols * CP;                // [kDsmWarps][RX]
  float2* twx = xr + kDsmWarps * RX;               // [k1][t] = W_256^(t k1)
  float2* w32x = twx + M;                          // [c][k2'] = W_256^(8 c k2')
  float2* tw2 = w32x + 32;                         // W_512^k, k <= 256
  float2* twy = tw2 + (M + 1);                     // [k1][t] = W_NY^(t k1)
  float2* w32y = twy + NY;                         // [c][k2'] = W_NY^(R1 c k2')
  const StageDesc& X = DIR < 0 ? s1 : s2;
  const StageDesc& Y = DIR < 0 ? s2 : s1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k1x = lane / CX, cx = lane % CX;
  const int mx = (cx >> 1) + 2 * (cx & 1);
  const uint32_t rank = cluster_cta_rank();
  const uint32_t col_s = smem_u32(col);
  pdl_launch_next();
  // twiddles: the x stage's natural table is W_512^m (the real kinds' length
  // 2 M), so W_256^j = W_512^(2 j)
  for (int i = threadIdx.x; i < M; i += kDsmThreads) twx[i] = X.twn[2 * ((i & 31) * (i >> 5))];
  if (threadIdx.x < 32) w32x[threadIdx.x] = X.twn[2 * ((R1X * (threadIdx.x / R1X) * (threadIdx.x % R1X)) % M)];
  for (int i = threadIdx.x; i <= M; i += kDsmThreads) tw2[i] = X.tw2[i];
  warp_load_twiddles<NY, kDsmThreads>(twy, w32y, Y);
  __syncthreads();
  pdl_wait_prev();
  cluster_barrier();  // every CTA of the cluster runs before any cluster access
  const long long planes = (long long)X.batch * X.n_outer;
  const long long nclusters = gridDim.x / kDsmCta;
  for (long long plane = blockIdx.x / kDsmCta; plane < planes; plane += nclusters) {
    const long long b = plane / X.n_outer, z = plane % X.n_outer;
    float2* wr = xr + warp * RX;  // this warp's x-stage region
    float2* cw = col + warp * CP; // this warp's column (y stage)
    if constexpr (DIR < 0) {
      // ---- (A) x stage: R2C rows, scattered to the column owners
      const float2* gin = X.in + b * X.in_b + z * X.in_o;
      float2 v[G::kRowTiles][R1X];
#pragma unroll
      for (int t = 0; t < G::kRowTiles; ++t) {
        const float2* src = gin + (long long)(rank * G::kRows + t * kDsmWarps + warp) * X.in_g;
#pragma unroll
        for (int i = 0; i < R1X; ++i) v[t][i] = ld_data(src + lane + 32 * i);
      }
#pragma unroll
      for (int t = 0; t < G::kRowTiles; ++t) {
        warp_steps12<M, -1>(v[t], wr, twx, w32x, lane);
        __syncwarp();
        warp_steps345<M, -1>(v[t], wr, w32x);
        __syncwarp();
#pragma unroll
        for (int k = 0; k < R1X; ++k) wr[k1x + R1X * k + R1X * R1X * mx] = v[t][k];
        __syncwarp();
        warp_r2c_post<M>(wr, tw2, X.interior);
        __syncthreads();  // the tile's 32 rows are complete
        const int y0 = rank * G::kRows + t * kDsmWarps;
#pragma unroll
        for (int u = 0; u < M * 16 / kDsmThreads; ++u) {
          const int it = threadIdx.x + u * kDsmThreads;
          const int pp = it & 15, kx = it >> 4;
          const float2* r0 = xr + 2 * pp * RX;
          const float2* r1 = r0 + RX;
          const float4 val = kx == 0 ? make_float4(r0[0].x, r0[M].x, r1[0].x, r1[M].x) : cat2(r0[kx], r1[kx]);
          const uint32_t a = col_s + (uint32_t)(((kx % kDsmCols) * CP + y0 + 2 * pp) * (int)sizeof(float2));
          st_cluster4(cluster_map(a, (uint32_t)(kx / kDsmCols)), val);
        }
        __syncthreads();  // the regions are free for the next row tile
      }
      cluster_barrier();  // every CTA's columns are complete
      // ---- (B) y stage in place, then the rows of this CTA's 32 columns to HBM
      dsm_column_fft<NY, -1>(cw, twy, w32y, Y.scale);
      float2* spare = xr;  // the bin-256 column (CTA 0)
      if (rank == 0 && warp == 0) {
        for (int k = lane; k <= NY / 2; k += 32) {
          const int km = (NY - k) & (NY - 1);
          const float2 zk = cw[k], zm = cw[km];
          const float2 a = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
          const float2 bb = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
          cw[k] = a;
          cw[km] = cconj(a);
          spare[k] = bb;
          spare[km] = cconj(bb);
        }
      }
      __syncthreads();
      float2* gout = Y.out + b * Y.out_b + z * Y.out_o + (long long)rank * kDsmCols * Y.out_g;
#pragma unroll 4
      for (int u = 0; u < NY * kDsmCols / kDsmThreads; ++u) {
        // half-warps along 16 columns of one row; the two halves take rows ky, ky + 1
        const int it = threadIdx.x + u * kDsmThreads;
        const int jl = it & 15, r = (it >> 4) & 1, rest = it >> 5;
        const int j = jl + 16 * (rest & 1), ky = 2 * (rest >> 1) + r;
        st_data(gout + (long long)ky * Y.out_n + (long long)j * Y.out_g, col[j * CP + ky]);
      }
      if (rank == 0)
        for (int ky = threadIdx.x; ky < NY; ky += kDsmThreads)
          st_data(gout + (long long)ky * Y.out_n + (long long)M * Y.out_g, spare[ky]);
      cluster_barrier();  // the column buffers are free for the next plane
    } else {
      // ---- (A) y stage: this CTA's 32 columns of the spectrum, transformed in place
      const float2* gin = Y.in + b * Y.in_b + z * Y.in_o;
      {
        constexpr int U = NY * kDsmCols / kDsmThreads;
        float2 lv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int it = threadIdx.x + u * kDsmThreads;
          const int jl = it & 15, r = (it >> 4) & 1, rest = it >> 5;
          const int j = jl + 16 * (rest & 1), ky = 2 * (rest >> 1) + r;
          lv[u] = ld_data(gin + (long long)ky * Y.in_n + (long long)(rank * kDsmCols + j) * Y.in_g);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int it = threadIdx.x + u * kDsmThreads;
          const int jl = it & 15, r = (it >> 4) & 1, rest = it >> 5;
          col[(jl + 16 * (rest & 1)) * CP + 2 * (rest >> 1) + r] = lv[u];
        }
      }
      __syncthreads();
      if (rank == 0 && warp == 0) {
        // column 0 <- Ah + i Bh of the columns kx = 0 (a, in column 0) and kx = 256 (b, from HBM)
        for (int k = lane; k <= NY / 2; k += 32) {
          const int km = (NY - k) & (NY - 1);
          const float2 ak = cw[k], am = cw[km];
          const float2 bk = ld_data(gin + (long long)k * Y.in_n + (long long)M * Y.in_g);
          const float2 bm = ld_data(gin + (long long)km * Y.in_n + (long long)M * Y.in_g);
          const float2 ah = make_float2(0.5f * (ak.x + am.x), 0.5f * (ak.y - am.y));
          const float2 bh = make_float2(0.5f * (bk.x + bm.x), 0.5f * (bk.y - bm.y));
          cw[k] = make_float2(ah.x - bh.y, ah.y + bh.x);
          cw[km] = make_float2(ah.x + bh.y, -ah.y + bh.x);
        }
        __syncwarp();
      }
      dsm_column_fft<NY, 1>(cw, twy, w32y, Y.scale);
      cluster_barrier();  // every CTA's columns are transformed
      // ---- (B) x stage: gather the rows' bins, C2R merge, transform, real rows to HBM
      float2* gout = X.out + b * X.out_b + z * X.out_o;
#pragma unroll 1
      for (int t = 0; t < G::kRowTiles; ++t) {
        const int y0 = rank * G::kRows + t * kDsmWarps;
        constexpr int UG = M * 16 / kDsmThreads;
        float4 gv[UG];
#pragma unroll
        for (int u = 0; u < UG; ++u) {
          const int it = threadIdx.x + u * kDsmThreads;
          const int pp = it & 15, kx = it >> 4;
          const uint32_t a = col_s + (uint32_t)(((kx % kDsmCols) * CP + y0 + 2 * pp) * (int)sizeof(float2));
          gv[u] = ld_cluster4(cluster_map(a, (uint32_t)(kx / kDsmCols)));
        }
#pragma unroll
        for (int u = 0; u < UG; ++u) {
          const int it = threadIdx.x + u * kDsmThreads;
          const int pp = it & 15, kx = it >> 4;
          const float4 val = gv[u];
          float2* r0 = xr + 2 * pp * RX;
          float2* r1 = r0 + RX;
          if (kx == 0) {
            r0[0] = make_float2(val.x, 0.f);
            r0[M] = make_float2(val.y, 0.f);
            r1[0] = make_float2(val.z, 0.f);
            r1[M] = make_float2(val.w, 0.f);
          } else {
            r0[kx] = lo2(val);
            r1[kx] = hi2(val);
          }
        }
        __syncthreads();
        warp_c2r_pre<M>(wr, tw2, X.interior);
        __syncwarp();
        float2 v[R1X];
#pragma unroll
        for (int i = 0; i < R1X; ++i) v[i] = wr[lane + 32 * i];
        __syncwarp();
        warp_steps12<M, 1>(v, wr, twx, w32x, lane);
        __syncwarp();
        warp_steps345<M, 1>(v, wr, w32x);
        float2* dst = gout + (long long)(y0 + warp) * X.out_g;
#pragma unroll
        for (int k = 0; k < R1X; ++k) st_data(dst + k1x + R1X * k + R1X * R1X * mx, cscale(v[k], X.scale));
        __syncthreads();  // the regions are free for the next row tile's gather
      }
      cluster_barrier();  // every CTA has read the column buffers
    }
  }
}

template <int NY, int DIR>
PlaneDsmKernel make_plane_dsm_entry() {
  return PlaneDsmKernel{NY, DIR, reinterpret_cast<const void*>(&plane_dsm_kernel<NY, DIR>), kDsmThreads,
                        plane_dsm_smem_bytes<NY>()};
}

}  // namespace gbfft
