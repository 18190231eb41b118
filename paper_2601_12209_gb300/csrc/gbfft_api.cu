// Host side of the C ABI declared in include/gbfft.h: plans, stage
// descriptors of the pencil and slab pipelines, persistent-launch counters, kernel
// dispatch.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/gbfft.h"
#include "gbfft_kernels.cuh"
#include "gbfft_many.cuh"
#include "gbfft_plane.cuh"
#include "gbfft_plane_dsm.cuh"
#include "gbfft_prefetch.cuh"
#include "gbfft_warp.cuh"

namespace gbfft {

void register_stage_group_0(std::vector<StageKernel>&);
void register_stage_group_1(std::vector<StageKernel>&);
void register_stage_group_2(std::vector<StageKernel>&);
void register_stage_group_3(std::vector<StageKernel>&);
void register_stage_group_4(std::vector<StageKernel>&);
void register_stage_group_5(std::vector<StageKernel>&);
void register_stage_group_6(std::vector<StageKernel>&);
void register_stage_group_7(std::vector<StageKernel>&);
void register_split_group_0(std::vector<StageKernel>&);
void register_split_group_1(std::vector<StageKernel>&);
void register_split_group_2(std::vector<StageKernel>&);
void register_split_group_3(std::vector<StageKernel>&);
void register_tc5_group_0(std::vector<StageKernel>&);
void register_tc5_group_1(std::vector<StageKernel>&);
void register_persistent_group_0(std::vector<PersistentKernel>&);
void register_persistent_group_1(std::vector<PersistentKernel>&);
void register_tma_group_0(std::vector<TmaKernel>&);
void register_tma_group_1(std::vector<TmaKernel>&);
void register_tma_group_2(std::vector<TmaKernel>&);
void register_plane_group_0(std::vector<PlaneKernel>&);
void register_plane_dsm_group_0(std::vector<PlaneDsmKernel>&);
void register_warp_group_0(std::vector<WarpKernel>&);
void register_warp_group_1(std::vector<WarpKernel>&);
void register_prefetch_group_0(std::vector<PrefetchKernel>&);

std::vector<PrefetchKernel>& prefetch_registry() {
  static std::vector<PrefetchKernel> v;
  return v;
}

std::vector<WarpKernel>& warp_registry() {
  static std::vector<WarpKernel> v;
  return v;
}

std::vector<PlaneKernel>& plane_registry() {
  static std::vector<PlaneKernel> v;
  return v;
}
std::vector<PlaneDsmKernel>& plane_dsm_registry() {
  static std::vector<PlaneDsmKernel> v;
  return v;
}
std::vector<StageKernel>& stage_registry() {
  static std::vector<StageKernel> v;
  return v;
}
std::vector<PersistentKernel>& persistent_registry() {
  static std::vector<PersistentKernel> v;
  return v;
}
std::vector<TmaKernel>& tma_registry() {
  static std::vector<TmaKernel> v;
  return v;
}

static std::once_flag g_reg_once;
static void ensure_registry() {
  std::call_once(g_reg_once, [] {
    auto& s = stage_registry();
    register_stage_group_0(s);
    register_stage_group_1(s);
    register_stage_group_2(s);
    register_stage_group_3(s);
    register_stage_group_4(s);
    register_stage_group_5(s);
    register_stage_group_6(s);
    register_stage_group_7(s);
    register_split_group_0(s);
    register_split_group_1(s);
    register_split_group_2(s);
    register_split_group_3(s);
    register_tc5_group_0(s);
    register_tc5_group_1(s);
    auto& p = persistent_registry();
    register_persistent_group_0(p);
    register_persistent_group_1(p);
    auto& t = tma_registry();
    register_tma_group_0(t);
    register_tma_group_1(t);
    register_tma_group_2(t);
    register_plane_group_0(plane_registry());
    register_plane_dsm_group_0(plane_dsm_registry());
    register_warp_group_0(warp_registry());
    register_warp_group_1(warp_registry());
    register_prefetch_group_0(prefetch_registry());
  });
}

// Host-side mirror of make_radices (device code is not callable here at
// run time for a runtime n).
static int host_radices(int n, int* out, int cap) {
  if (n < 2) return -1;
  int m = n, a = 0, cnt = 0;
  int tmp[16];
  while (m % 2 == 0) {
    ++a;
    m /= 2;
  }
  if (a > 0) {
    int passes = (a + 3) / 4;
    int base = a / passes, extra = a % passes;
    for (int i = 0; i < passes; ++i) tmp[cnt++] = 1 << (base + (i < extra ? 1 : 0));
  }
  while (m % 3 == 0) {
    tmp[cnt++] = 3;
    m /= 3;
  }
  while (m % 5 == 0) {
    tmp[cnt++] = 5;
    m /= 5;
  }
  if (m != 1) return -1;
  for (int i = 0; i < cnt && i < cap; ++i) out[i] = tmp[i];
  return cnt;
}

// Lengths with tensor-core passes: a radix-16 pass and whole warps (length 16
// alone runs as a 16-thread block and keeps the FP32 butterflies).
static bool split_capable(int L) {
  const Radices R = make_radices(L);
  bool r16 = false;
  for (int i = 0; i < R.n; ++i) r16 |= R.r[i] == 16;
  return r16 && threads_for(L) % 32 == 0;
}

// Lengths without tensor-core passes run the same FP32 arithmetic in every
// precision mode, so a split-precision request takes the FP32 kernel; a
// 5th-generation tensor-core request for a length whose radix-16 butterflies
// do not fill 128-row operand tiles takes the warp-level (mma.sync) kernel of
// the same operand type.
static const StageKernel* find_stage(int L, int dir, int kind, int prec = kPrecFP32) {
  ensure_registry();
  if (prec != kPrecFP32 && !split_capable(L)) prec = kPrecFP32;
  for (int attempt = 0; attempt < 2; ++attempt) {
    for (const auto& k : stage_registry())
      if (k.L == L && k.dir == dir && k.kind == kind && k.prec == prec) return &k;
    if (!prec_is_tc5(prec)) break;
    prec = prec_mma_sync(prec);
  }
  return nullptr;
}

static bool stage_supported(int L) { return find_stage(L, -1, kPlain) != nullptr; }

static const TmaKernel* find_tma(int L, int dir, int kind, int src) {
  ensure_registry();
  for (const auto& k : tma_registry())
    if (k.L == L && k.dir == dir && k.kind == kind && k.src == src) return &k;
  return nullptr;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (the
// library links only the CUDA runtime).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
    else
      cudaGetLastError();
  });
  return fn;
}

// Tensor map of a stage's input for the TMA kernel, or false when the layout
// cannot be described (a stride or the base not a multiple of 16 bytes).
//   row side:    dims {2 n_in floats, pencils, outer, batch}, box {32, 16, 1, 1}
//   column side: dims {2 pencils floats, n_in, outer, batch}, box {32, kColBoxN, 1, 1}
static bool encode_input_map(const StageDesc& d, int src, CUtensorMap* m) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  if ((reinterpret_cast<uintptr_t>(d.in) & 15) != 0) return false;
  cuuint64_t dims[4];
  long long strides_el[3];
  cuuint32_t box[4] = {32, 0, 1, 1};
  cuuint32_t es[4] = {1, 1, 1, 1};
  if (src == 1) {
    if (d.in_mode != kRow) return false;
    dims[0] = 2ull * d.n_in;
    dims[1] = (cuuint64_t)d.n_group;
    strides_el[0] = d.in_g;
    box[1] = kTileP;
  } else {
    if (d.in_mode != kCol) return false;
    dims[0] = 2ull * d.n_group;
    dims[1] = (cuuint64_t)d.n_in;
    strides_el[0] = d.in_n;
    box[1] = kColBoxN;
  }
  dims[2] = (cuuint64_t)d.n_outer;
  dims[3] = (cuuint64_t)d.batch;
  strides_el[1] = d.in_o;
  strides_el[2] = d.in_b;
  cuuint64_t strides[3];
  for (int i = 0; i < 3; ++i) {
    long long bytes = strides_el[i] * 8;
    if (dims[i + 1] == 1) bytes = std::max<long long>(16, (bytes + 15) / 16 * 16);  // unused coordinate
    if (bytes <= 0 || bytes % 16 != 0 || bytes >= (1LL << 40)) return false;
    strides[i] = (cuuint64_t)bytes;
  }
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float2*>(d.in), dims, strides, box, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Per-device launch facts of one kernel (max dynamic smem set, blocks per SM).
struct LaunchInfo {
  int blocks_per_sm = 0;
  bool ready = false;
};
static std::mutex g_launch_mu;
static std::map<std::tuple<int, const void*, size_t>, LaunchInfo> g_launch;

static cudaError_t launch_info(const void* fn, int threads, size_t smem, int* blocks_per_sm) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_launch_mu);
  LaunchInfo& li = g_launch[std::make_tuple(dev, fn, smem)];
  if (!li.ready) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem);
    if (e != cudaSuccess) return e;
    li.blocks_per_sm = std::max(nb, 1);
    li.ready = true;
  }
  *blocks_per_sm = li.blocks_per_sm;
  return cudaSuccess;
}

static int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return std::max(n, 1);
}

}  // namespace gbfft

using namespace gbfft;

// ----------------------------------------------------------------- the plan

enum Pipe { kPipeFwd = 0, kPipeInv = 1, kPipePoisson = 2, kNumPipes = 3 };

struct gbfft_plan_s {
  int nx, ny, nz, batch, kind, dtype;
  unsigned flags;
  int device;
  int nxc, Lx, rowA;  // spectrum x bins, x transform length, complex per input row
  long long Nc, NA;   // spectrum / input float2 elements per batch entry
  // twiddle tables (device)
  float2 *tw_x = nullptr, *tw_y = nullptr, *tw_z = nullptr, *tw2 = nullptr;
  float2 *twn_x = nullptr, *twn_y = nullptr, *twn_z = nullptr;  // natural W_L^m tables per axis
  float2* twn_real = nullptr;  // W_nx^m, m < nx: the real x stages' two-for-one transforms (R2C plans)
  float2 *tw4_x = nullptr, *tw4_y = nullptr, *tw4_z = nullptr;  // W_4L^k, k <= L: DCT / DST stages per axis
  // workspace
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = false;
  int n_ws = 0;
  // persistent launch state
  Control* ctl = nullptr;
  unsigned int* counters = nullptr;
  size_t counters_words = 0;
  // end-to-end host path
  void* h_in_dev = nullptr;
  void* h_out_dev = nullptr;
  size_t h_in_bytes = 0, h_out_bytes = 0;
  cudaStream_t h_stream = nullptr;
  // chunked host-buffer execution: slabs of the first and last stages, their copies on h_stream, the
  // stages on h_stream2, ordered by events
  int host_chunks = 1;
  cudaStream_t h_stream2 = nullptr;
  cudaEvent_t h_ev[32] = {};
  // autotuned launch choice per pipeline (forward, inverse, Poisson)
  struct Tuning {
    bool tuned = false;
    bool persistent = false;
    unsigned tma_mask = 0;  // bit s: stage s uses the tensor-copy kernel
    unsigned plane_mask = 0;  // bit s: stages s and s+1 run as one fused plane launch
    unsigned warp_mask = 0;   // bit s: stage s runs the warp-per-pencil kernel
    unsigned prefetch_mask = 0;  // bit s: stage s runs the cp.async prefetch C2R kernel
    int persistent_tiles = 1;    // persistent launch: consecutive tiles per ticket (1, 2, 4)
    int plane_cx = 0;         // CTAs per plane cluster of the fused launches (0: by plane size)
    bool plane_dsm = false;   // fused plane launches keep the intermediate in distributed shared memory
    float ms = 0.f;         // measured time of the chosen launch(es)
    float stage_ms[kMaxStages] = {0.f, 0.f, 0.f, 0.f, 0.f};
  } tune[3];
  // optional per-stage event timing inside exec calls
  bool time_stages = false;
  struct TimedCall {
    int pipe, nev;
    cudaEvent_t ev[kMaxStages + 1];
  };
  std::vector<TimedCall> timed;
};

static int cuda_err(cudaError_t e) { return e == cudaSuccess ? GBFFT_OK : GBFFT_ERR_CUDA; }

static bool is_r2c(const gbfft_plan_s* p) { return p->kind == GBFFT_R2C; }
static bool is_slab(const gbfft_plan_s* p) { return (p->flags & GBFFT_SLAB) != 0; }

static int gchunks(int n) { return (n + kTileP - 1) / kTileP; }

static StageDesc mk(const void* in, void* out, int L, int kind, int dir, int batch, int n_outer, int n_group,
                    long long ib, long long io, long long ig, long long in_, int im, long long ob, long long oo,
                    long long og, long long on_, int om, float scale, float interior, const float2* tw,
                    const float2* tw2) {
  StageDesc d;
  std::memset(&d, 0, sizeof(d));
  d.in = reinterpret_cast<const float2*>(in);
  d.out = reinterpret_cast<float2*>(out);
  d.in_b = ib;
  d.in_o = io;
  d.in_g = ig;
  d.in_n = in_;
  d.out_b = ob;
  d.out_o = oo;
  d.out_g = og;
  d.out_n = on_;
  d.batch = batch;
  d.n_outer = n_outer;
  d.n_group = n_group;
  d.n_gchunks = gchunks(n_group);
  d.n_tiles = (long long)batch * n_outer * d.n_gchunks;
  d.L = L;
  d.n_in = kind == kC2RPre ? L + 1 : L;
  d.n_out = kind == kR2CPost ? L + 1 : L;
  d.in_mode = im;
  d.out_mode = om;
  d.kind = kind;
  d.dir = dir;
  d.scale = scale;
  d.interior = interior;
  d.tw = tw;
  d.tw2 = tw2;
  d.tw_len = tw_table_len(L);
  d.dep_rule = kDepNone;
  return d;
}

static void dep(StageDesc& d, int rule, const StageDesc& prev) {
  d.dep_rule = rule;
  d.prev_n_outer = prev.n_outer;
  d.prev_n_gchunks = prev.n_gchunks;
}

struct Pipeline {
  StageDesc st[kMaxStages];
  long long in_cap[kMaxStages];   // float2 capacity of the buffer each stage reads
  long long out_cap[kMaxStages];  // ... and writes (-1: unknown, not checked)
  int n = 0;
};

// A buffer of the pipeline and its capacity in float2 elements.
struct Buf {
  void* p;
  long long cap;
};

// Largest float2 offset + 1 a stage reads / writes (all strides are positive).
static long long read_extent(const StageDesc& d) {
  return (long long)(d.batch - 1) * d.in_b + (long long)(d.n_outer - 1) * d.in_o +
         (long long)(d.n_group - 1) * d.in_g + (long long)(d.n_in - 1) * d.in_n + 1;
}
static long long write_extent(const StageDesc& d) {
  return (long long)(d.batch - 1) * d.out_b + (long long)(d.n_outer - 1) * d.out_o +
         (long long)(d.n_group - 1) * d.out_g + (long long)(d.n_out - 1) * d.out_n + 1;
}

// Stage descriptors of one operation. Buffers: in, out, W1, W2 (workspace).
// Layouts (float2 units; nxc = spectrum x bins):
//   A natural input  [b][z][y][rowA]   B [b][z][kx][y]   C [b][kx][y][z]
//   S natural spectrum [b][z][y][kx]
// r2r (optional): per axis x, y, z GBFFT_R2R_NONE (Fourier), GBFFT_R2R_DCT or
// GBFFT_R2R_DST; those axes' stages become the real-to-real kinds (forward
// op: type II, inverse op: type III, whose 2L factor joins the 1/N scale).
static Pipeline build_pipeline(const gbfft_plan_s* p, int pipe, int op, Buf bin, Buf bout, Buf b1, Buf b2,
                               const int* r2r = nullptr) {
  Pipeline P;
  const void* in = bin.p;
  void* out = bout.p;
  void* W1 = b1.p;
  void* W2 = b2.p;
  // capacity of whichever buffer a stage uses (matched by role, not address)
  auto cap_of = [&](int role) -> long long {
    switch (role) {
      case 0: return bin.cap;
      case 1: return bout.cap;
      case 2: return b1.cap;
      default: return b2.cap;
    }
  };
  const int B = p->batch, nx = p->nx, ny = p->ny, nz = p->nz, nxc = p->nxc, Lx = p->Lx, rowA = p->rowA;
  const long long Nc = p->Nc, NA = p->NA;
  const bool r2c = is_r2c(p);
  const float invN = (float)(1.0 / ((double)nx * (double)ny * (double)nz));
  const int kx_kind_f = r2c ? kR2CPost : kPlain;
  const int kx_kind_i = r2c ? kC2RPre : kPlain;
  // roles: 0 in, 1 out, 2 W1, 3 W2
  auto add = [&](const StageDesc& d, int rin, int rout) {
    P.st[P.n] = d;
    P.in_cap[P.n] = cap_of(rin);
    P.out_cap[P.n] = cap_of(rout);
    ++P.n;
  };
  if (pipe == kPipeFwd) {
    const float interior = (op == GBFFT_OP_INVERSE_ADJOINT) ? 2.f : 1.f;
    const float scale = (op == GBFFT_OP_INVERSE_ADJOINT) ? invN : 1.f;
    if (!is_slab(p)) {
      StageDesc X = mk(in, out, Lx, kx_kind_f, -1, B, nz, ny, NA, (long long)rowA * ny, rowA, 1, kRow, Nc,
                       (long long)nxc * ny, 1, ny, kCol, 1.f, r2c ? interior : 1.f, p->tw_x, p->tw2);
      StageDesc Y = mk(out, W1, ny, kPlain, -1, B, nxc, nz, Nc, ny, (long long)nxc * ny, 1, kRow, Nc,
                       (long long)ny * nz, 1, nz, kCol, 1.f, 1.f, p->tw_y, nullptr);
      dep(Y, kDepGroup, X);
      StageDesc Z;
      if (p->flags & GBFFT_TRANSPOSED_OUT)
        Z = mk(W1, out, nz, kPlain, -1, B, ny, nxc, Nc, nz, (long long)ny * nz, 1, kRow, Nc, nz,
               (long long)ny * nz, 1, kRow, scale, 1.f, p->tw_z, nullptr);
      else
        Z = mk(W1, out, nz, kPlain, -1, B, ny, nxc, Nc, nz, (long long)ny * nz, 1, kRow, Nc, nxc, 1,
               (long long)nxc * ny, kCol, scale, 1.f, p->tw_z, nullptr);
      dep(Z, kDepGroup, Y);
      add(X, 0, 1);
      add(Y, 1, 2);
      add(Z, 2, 1);
    } else {
      StageDesc X = mk(in, out, Lx, kx_kind_f, -1, B, nz, ny, NA, (long long)rowA * ny, rowA, 1, kRow, Nc,
                       (long long)nxc * ny, nxc, 1, kRow, 1.f, r2c ? interior : 1.f, p->tw_x, p->tw2);
      StageDesc Y = mk(out, out, ny, kPlain, -1, B, nz, nxc, Nc, (long long)nxc * ny, 1, nxc, kCol, Nc,
                       (long long)nxc * ny, 1, nxc, kCol, 1.f, 1.f, p->tw_y, nullptr);
      dep(Y, kDepOuter, X);
      StageDesc Z = mk(out, out, nz, kPlain, -1, B, ny, nxc, Nc, nxc, 1, (long long)nxc * ny, kCol, Nc, nxc, 1,
                       (long long)nxc * ny, kCol, scale, 1.f, p->tw_z, nullptr);
      dep(Z, kDepSameGchunk, Y);
      add(X, 0, 1);
      add(Y, 1, 1);
      add(Z, 1, 1);
    }
  } else if (pipe == kPipeInv) {
    const float interior = (op == GBFFT_OP_ADJOINT) ? 0.5f : 1.f;
    // the real-to-real inverses (DCT-III, DST-III) return 2 nz times the input along z
    const float scale = (op == GBFFT_OP_INVERSE) ? invN : 1.f;
    if (!is_slab(p)) {
      void* Cb = r2c ? W1 : out;
      void* Bb = r2c ? W2 : W1;
      StageDesc Z;
      if (p->flags & GBFFT_TRANSPOSED_OUT)
        Z = mk(in, Cb, nz, kPlain, +1, B, ny, nxc, Nc, nz, (long long)ny * nz, 1, kRow, Nc, nz,
               (long long)ny * nz, 1, kRow, 1.f, 1.f, p->tw_z, nullptr);
      else
        Z = mk(in, Cb, nz, kPlain, +1, B, ny, nxc, Nc, nxc, 1, (long long)nxc * ny, kCol, Nc, nz,
               (long long)ny * nz, 1, kRow, 1.f, 1.f, p->tw_z, nullptr);
      StageDesc Y = mk(Cb, Bb, ny, kPlain, +1, B, nxc, nz, Nc, (long long)ny * nz, 1, nz, kCol, Nc, ny,
                       (long long)nxc * ny, 1, kRow, 1.f, 1.f, p->tw_y, nullptr);
      dep(Y, kDepGchunkOfOuter, Z);
      StageDesc X = mk(Bb, out, Lx, kx_kind_i, +1, B, nz, ny, Nc, (long long)nxc * ny, 1, ny, kCol, NA,
                       (long long)rowA * ny, rowA, 1, kRow, scale, r2c ? interior : 1.f, p->tw_x, p->tw2);
      dep(X, kDepGchunkOfOuter, Y);
      add(Z, 0, r2c ? 2 : 1);
      add(Y, r2c ? 2 : 1, r2c ? 3 : 2);
      add(X, r2c ? 3 : 2, 1);
    } else {
      void* D = r2c ? W1 : out;
      StageDesc Z = mk(in, D, nz, kPlain, +1, B, ny, nxc, Nc, nxc, 1, (long long)nxc * ny, kCol, Nc, nxc, 1,
                       (long long)nxc * ny, kCol, 1.f, 1.f, p->tw_z, nullptr);
      StageDesc Y = mk(D, D, ny, kPlain, +1, B, nz, nxc, Nc, (long long)nxc * ny, 1, nxc, kCol, Nc,
                       (long long)nxc * ny, 1, nxc, kCol, 1.f, 1.f, p->tw_y, nullptr);
      dep(Y, kDepSameGchunk, Z);
      StageDesc X = mk(D, out, Lx, kx_kind_i, +1, B, nz, ny, Nc, (long long)nxc * ny, nxc, 1, kRow, NA,
                       (long long)rowA * ny, rowA, 1, kRow, scale, r2c ? interior : 1.f, p->tw_x, p->tw2);
      dep(X, kDepOuter, Y);
      add(Z, 0, r2c ? 2 : 1);
      add(Y, r2c ? 2 : 1, r2c ? 2 : 1);
      add(X, r2c ? 2 : 1, 1);
    }
  } else {  // Poisson (R2C plans); op 5: bounded z (Neumann walls, DCT-II / DCT-III along z)
    const int M = Lx;
    const bool bounded = op == 5;
    // DCT-III(DCT-II(x)) = 2 nz x; the x,y transforms contribute nx ny
    const float invNb = (float)(1.0 / (2.0 * (double)nx * (double)ny * (double)nz));
    if (!is_slab(p)) {
      StageDesc X = mk(in, W1, M, kR2CPost, -1, B, nz, ny, NA, (long long)M * ny, M, 1, kRow, Nc,
                       (long long)nxc * ny, 1, ny, kCol, 1.f, 1.f, p->tw_x, p->tw2);
      StageDesc Y = mk(W1, W2, ny, kPlain, -1, B, nxc, nz, Nc, ny, (long long)nxc * ny, 1, kRow, Nc,
                       (long long)ny * nz, 1, nz, kCol, 1.f, 1.f, p->tw_y, nullptr);
      dep(Y, kDepGroup, X);
      StageDesc PZ = bounded ? mk(W2, W2, nz, kPoissonZB, -1, B, ny, nxc, Nc, nz, (long long)ny * nz, 1, kRow, Nc,
                                  nz, (long long)ny * nz, 1, kRow, invNb, 1.f, p->tw_z, p->tw4_z)
                             : mk(W2, W2, nz, kPoissonZ, -1, B, ny, nxc, Nc, nz, (long long)ny * nz, 1, kRow, Nc, nz,
                                  (long long)ny * nz, 1, kRow, invN, 1.f, p->tw_z, nullptr);
      PZ.pz_nx = nx;
      PZ.pz_ny = ny;
      dep(PZ, kDepGroup, Y);
      StageDesc Yi = mk(W2, W1, ny, kPlain, +1, B, nxc, nz, Nc, (long long)ny * nz, 1, nz, kCol, Nc, ny,
                        (long long)nxc * ny, 1, kRow, 1.f, 1.f, p->tw_y, nullptr);
      dep(Yi, kDepGchunkOfOuter, PZ);
      StageDesc Xi = mk(W1, out, M, kC2RPre, +1, B, nz, ny, Nc, (long long)nxc * ny, 1, ny, kCol, NA,
                        (long long)M * ny, M, 1, kRow, 1.f, 1.f, p->tw_x, p->tw2);
      dep(Xi, kDepGchunkOfOuter, Yi);
      add(X, 0, 2);
      add(Y, 2, 3);
      add(PZ, 3, 3);
      add(Yi, 3, 2);
      add(Xi, 2, 1);
    } else {
      StageDesc X = mk(in, W1, M, kR2CPost, -1, B, nz, ny, NA, (long long)M * ny, M, 1, kRow, Nc,
                       (long long)nxc * ny, nxc, 1, kRow, 1.f, 1.f, p->tw_x, p->tw2);
      StageDesc Y = mk(W1, W1, ny, kPlain, -1, B, nz, nxc, Nc, (long long)nxc * ny, 1, nxc, kCol, Nc,
                       (long long)nxc * ny, 1, nxc, kCol, 1.f, 1.f, p->tw_y, nullptr);
      dep(Y, kDepOuter, X);
      StageDesc PZ = mk(W1, W1, nz, bounded ? kPoissonZB : kPoissonZ, -1, B, ny, nxc, Nc, nxc, 1,
                        (long long)nxc * ny, kCol, Nc, nxc, 1, (long long)nxc * ny, kCol, bounded ? invNb : invN, 1.f,
                        p->tw_z, bounded ? p->tw4_z : nullptr);
      PZ.pz_nx = nx;
      PZ.pz_ny = ny;
      dep(PZ, kDepSameGchunk, Y);
      StageDesc Yi = mk(W1, W1, ny, kPlain, +1, B, nz, nxc, Nc, (long long)nxc * ny, 1, nxc, kCol, Nc,
                        (long long)nxc * ny, 1, nxc, kCol, 1.f, 1.f, p->tw_y, nullptr);
      dep(Yi, kDepSameGchunk, PZ);
      StageDesc Xi = mk(W1, out, M, kC2RPre, +1, B, nz, ny, Nc, (long long)nxc * ny, nxc, 1, kRow, NA,
                        (long long)M * ny, M, 1, kRow, 1.f, 1.f, p->tw_x, p->tw2);
      dep(Xi, kDepOuter, Yi);
      add(X, 0, 2);
      add(Y, 2, 2);
      add(PZ, 2, 2);
      add(Yi, 2, 2);
      add(Xi, 2, 1);
    }
  }
  if (r2r && P.n == 3 && (pipe == kPipeFwd || pipe == kPipeInv)) {
    // stages in axis order x, y, z forward and z, y, x inverse
    const float2* tw4[3] = {p->tw4_x, p->tw4_y, p->tw4_z};
    for (int ax = 0; ax < 3; ++ax) {
      if (r2r[ax] != GBFFT_R2R_DCT && r2r[ax] != GBFFT_R2R_DST) continue;
      StageDesc& d = P.st[pipe == kPipeFwd ? ax : 2 - ax];
      const bool dct = r2r[ax] == GBFFT_R2R_DCT;
      d.kind = pipe == kPipeFwd ? (dct ? kDct2 : kDst2) : (dct ? kDct3 : kDst3);
      d.tw2 = tw4[ax];
    }
    if (pipe == kPipeInv) {
      int n_r2r = 0;
      for (int ax = 0; ax < 3; ++ax) n_r2r += (r2r[ax] == GBFFT_R2R_DCT || r2r[ax] == GBFFT_R2R_DST) ? 1 : 0;
      P.st[2].scale *= 1.f / (float)(1 << n_r2r);  // DCT-III(DCT-II(x)) = 2L x
    }
  }
  for (int s = 0; s < P.n; ++s) {
    StageDesc& d = P.st[s];
    if (d.kind == kPlain) d.prec = p->dtype;  // GBFFT_*_SPLIT* values equal the StagePrec values
    d.err = p->ctl ? &p->ctl->error : nullptr;
    d.twn = d.tw == p->tw_x ? p->twn_x : (d.tw == p->tw_y ? p->twn_y : (d.tw == p->tw_z ? p->twn_z : nullptr));
    if (d.kind == kR2CPost || d.kind == kC2RPre) d.twn = p->twn_real;  // length nx = 2 L
  }
  return P;
}

// ops 0-3: GBFFT_OP_*; 4, 5: Poisson (periodic, bounded z)
static int pipe_of(int op) {
  if (op == GBFFT_OP_FORWARD || op == GBFFT_OP_INVERSE_ADJOINT) return kPipeFwd;
  if (op == GBFFT_OP_INVERSE || op == GBFFT_OP_ADJOINT) return kPipeInv;
  return kPipePoisson;
}

// Counters of one stage: per (batch, outer), per (batch, outer/16), per
// (batch, group chunk), per batch, and one for the whole stage.
static size_t stage_counter_words(const StageDesc& d) {
  return (size_t)d.batch * d.n_outer + (size_t)d.batch * gchunks(d.n_outer) + (size_t)d.batch * d.n_gchunks +
         (size_t)d.batch + 1;
}

static size_t counter_words(const Pipeline& P) {
  size_t w = 0;
  for (int k = 0; k < P.n; ++k) w += stage_counter_words(P.st[k]);
  return w;
}

static const PersistentKernel* find_persistent(const Pipeline& P) {
  ensure_registry();
  for (int s = 0; s < P.n; ++s)
    if (P.st[s].prec != kPrecFP32) return nullptr;  // tensor-core passes run in stage launches only
  for (const auto& k : persistent_registry()) {
    bool all = true;
    for (int s = 0; s < P.n && all; ++s) {
      const int code = kcode(P.st[s].L, P.st[s].kind, P.st[s].dir);
      bool found = false;
      for (int i = 0; i < k.ncodes; ++i) found |= (k.codes[i] == code);
      all = found;
    }
    if (all) return &k;
  }
  return nullptr;
}

// Launch a stage kernel with programmatic stream serialization: it may start
// while the previous kernel in the stream drains (the kernel waits for that
// grid before it reads its input; see pdl_wait_prev).
static cudaError_t launch_stage_kernel(const void* fn, long long grid, int threads, void** args, size_t smem,
                                       cudaStream_t stream) {
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

// Internal launch flag: run the stage with the warp-per-pencil kernel where one
// is built (lengths 512 and 256 complex, the length-256 real x stages; FP32).
constexpr unsigned kUseWarpKernel = 1u << 30;

// Internal launch flag: run a C2R x stage with the cp.async prefetch kernel
// (column-side half spectrum in, real rows out; FP32).
constexpr unsigned kUsePrefetchKernel = 1u << 29;

// Launch flags of a stage from its tuning bits (tensor-copy, warp-per-pencil,
// C2R prefetch kernel).
static unsigned stage_flags(bool tma, bool warp, bool prefetch) {
  return (tma ? 0u : GBFFT_NO_TMA) | (warp ? kUseWarpKernel : 0u) | (prefetch ? kUsePrefetchKernel : 0u);
}

static const PrefetchKernel* find_prefetch(const StageDesc& d) {
  if (d.prec != kPrecFP32 || d.kind != kC2RPre || d.dir < 0 || !d.tw2) return nullptr;
  if (d.in_mode != kCol || d.out_mode != kRow || static_cast<const void*>(d.in) == static_cast<const void*>(d.out))
    return nullptr;
  ensure_registry();
  for (const auto& k : prefetch_registry())
    if (k.L == d.L) return &k;
  return nullptr;
}

static const WarpKernel* find_warp(const StageDesc& d) {
  if (d.prec != kPrecFP32 || !d.twn) return nullptr;
  if (d.kind != kPlain && d.kind != kR2CPost && d.kind != kC2RPre) return nullptr;
  if (d.kind == kR2CPost && d.in_mode != kRow) return nullptr;   // the split reads row-side pairs
  if (d.kind == kC2RPre && d.out_mode != kRow) return nullptr;   // the merge writes row-side pairs
  if ((d.kind == kR2CPost || d.kind == kC2RPre) && !d.tw2) return nullptr;
  ensure_registry();
  // a kernel specialised for the stage's layout, else one for any layout
  const int io = warp_io(d.in_mode, d.out_mode);
  const WarpKernel* any = nullptr;
  for (const auto& k : warp_registry())
    if (k.L == d.L && k.dir == d.dir && k.kind == d.kind) {
      if (k.io == io) return &k;
      if (k.io < 0 && !any) any = &k;
    }
  return any;
}

// Warp-per-pencil launches: when the column side of a stage is linear in
// m = o * n_group + g (its outer stride is n_group group strides, as in the
// natural spectrum [z][y][kx] read or written by the z stages), the outer and
// group indices merge into one group axis of n_outer * n_group pencils. The
// 16-pencil chunks then tile that axis with no ragged chunk per outer index
// (nx/2 + 1 spectrum rows leave one of 17 chunks nearly empty otherwise), and
// every chunk's 16 elements fill one aligned 128-byte line instead of
// straddling two. A row side, if any, addresses its pencils through
// (m / n_group, m % n_group).
static void merge_pencils(StageDesc& d) {
  if (d.n_outer <= 1) return;
  const bool cin = d.in_mode == kCol, cout = d.out_mode == kCol;
  if (!cin && !cout) return;
  if (cin && d.in_o != (long long)d.n_group * d.in_g) return;
  if (cout && d.out_o != (long long)d.n_group * d.out_g) return;
  const long long m_total = (long long)d.n_outer * d.n_group;
  if (m_total > 0x7FFFFFFFLL) return;
  if (!cin) {
    d.m_split = d.n_group;
    d.split_o = d.in_o;
    d.split_g = d.in_g;
    d.in_g = 0;
  } else if (!cout) {
    d.m_split = d.n_group;
    d.split_o = d.out_o;
    d.split_g = d.out_g;
    d.out_g = 0;
  }
  d.in_o = 0;
  d.out_o = 0;
  d.n_outer = 1;
  d.n_group = (int)m_total;
  d.n_gchunks = gchunks(d.n_group);
  d.n_tiles = (long long)d.batch * d.n_gchunks;
}

// Launch one stage: the warp-per-pencil kernel when asked for and built, the
// TMA kernel when one exists for the stage and its input layout can be
// described by a tensor map, else the load/store kernel.
static int launch_stage(const StageDesc& d, cudaStream_t stream, unsigned flags = 0, int* err = nullptr) {
  if (d.n_tiles == 0) return GBFFT_OK;
  if (flags & kUsePrefetchKernel) {
    if (const PrefetchKernel* pk = find_prefetch(d)) {
      int bpsm = 1;
      cudaError_t e = launch_info(pk->fn, pk->threads, pk->smem, &bpsm);
      if (e != cudaSuccess) return GBFFT_ERR_CUDA;
      const long long grid = std::min<long long>(d.n_tiles, (long long)sm_count() * bpsm);
      StageDesc dd = d;
      void* args[] = {&dd};
      return cuda_err(launch_stage_kernel(pk->fn, grid, pk->threads, args, pk->smem, stream));
    }
  }
  if (flags & kUseWarpKernel) {
    if (const WarpKernel* wk = find_warp(d)) {
      int bpsm = 1;
      cudaError_t e = launch_info(wk->fn, wk->threads, wk->smem, &bpsm);
      if (e != cudaSuccess) return GBFFT_ERR_CUDA;
      StageDesc dd = d;
      if (d.kind == kPlain) merge_pencils(dd);
      const long long grid = std::min<long long>(dd.n_tiles, (long long)sm_count() * bpsm);
      void* args[] = {&dd};
      return cuda_err(launch_stage_kernel(wk->fn, grid, wk->threads, args, wk->smem, stream));
    }
  }
  if (!(flags & GBFFT_NO_TMA) && err && d.kind != kIdentity && d.prec == kPrecFP32) {
    const int src = d.in_mode == kRow ? 1 : 2;
    const TmaKernel* tk = find_tma(d.L, d.dir, d.kind, src);
    alignas(64) CUtensorMap map;
    if (tk && encode_input_map(d, src, &map)) {
      int bpsm = 1;
      cudaError_t e = launch_info(tk->fn, tk->threads, tk->smem, &bpsm);
      if (e != cudaSuccess) return GBFFT_ERR_CUDA;
      long long grid = std::min<long long>(d.n_tiles, (long long)sm_count() * bpsm);
      StageDesc dd = d;
      long long timeout_ns = 2000000000LL;
      void* args[] = {&map, &dd, &err, &timeout_ns};
      e = launch_stage_kernel(tk->fn, grid, tk->threads, args, tk->smem, stream);
      return cuda_err(e);
    }
  }
  const StageKernel* k = find_stage(d.L, d.dir, d.kind, d.prec);
  if (!k) return GBFFT_ERR_UNSUPPORTED_SIZE;
  int bpsm = 1;
  cudaError_t e = launch_info(k->fn, k->threads, k->smem, &bpsm);
  if (e != cudaSuccess) return GBFFT_ERR_CUDA;
  if (!k->loops && d.n_tiles > 0x7FFFFFFFLL) return GBFFT_ERR_INVALID_ARG;
  long long grid = k->loops ? std::min<long long>(d.n_tiles, (long long)sm_count() * bpsm) : d.n_tiles;
  StageDesc dd = d;
  void* args[] = {&dd};
  e = launch_stage_kernel(k->fn, grid, k->threads, args, k->smem, stream);
  return cuda_err(e);
}

namespace gbfft {
// Launch one stage through the registry; used by the allocation-free entry
// point in gbfft_static.cu.
int launch_stage_external(const StageDesc& d, cudaStream_t stream) {
  return launch_stage(d, stream, GBFFT_NO_TMA, nullptr);
}
}  // namespace gbfft

static int ensure_workspace(gbfft_plan_s* p) {
  if (p->n_ws == 0 || p->ws) return GBFFT_OK;
  size_t need = 0;
  gbfft_workspace_size(p, &need);
  if (cudaMalloc(&p->ws, need) != cudaSuccess) {
    p->ws = nullptr;
    cudaGetLastError();
    return GBFFT_ERR_ALLOC;
  }
  p->ws_bytes = need;
  p->ws_owned = true;
  return GBFFT_OK;
}

static size_t spectrum_bytes(const gbfft_plan_s* p) {
  size_t b = (size_t)p->Nc * (size_t)p->batch * sizeof(float2);
  return (b + 255) & ~(size_t)255;
}

// Host-side bounds check of every stage against the buffers it touches: an
// indexing error becomes GBFFT_ERR_INVALID_ARG instead of a launch.
static int validate(const Pipeline& P) {
  for (int s = 0; s < P.n; ++s) {
    const StageDesc& d = P.st[s];
    if (d.n_tiles <= 0 || d.batch < 1 || d.n_outer < 1 || d.n_group < 1) return GBFFT_ERR_INVALID_ARG;
    if (d.in_mode == kRow ? d.in_n != 1 : d.in_g != 1) return GBFFT_ERR_INVALID_ARG;
    if (d.out_mode == kRow ? d.out_n != 1 : d.out_g != 1) return GBFFT_ERR_INVALID_ARG;
    if (P.in_cap[s] >= 0 && read_extent(d) > P.in_cap[s]) return GBFFT_ERR_INVALID_ARG;
    if (P.out_cap[s] >= 0 && write_extent(d) > P.out_cap[s]) return GBFFT_ERR_INVALID_ARG;
    if (!d.in || !d.out || !d.tw) return GBFFT_ERR_INVALID_ARG;
    if ((d.kind == kR2CPost || d.kind == kC2RPre) && !d.tw2) return GBFFT_ERR_INVALID_ARG;
  }
  return GBFFT_OK;
}

// Events around a pipeline's launches when per-stage timing is on (one event
// before the first launch and one after each launch, on the launching stream).
static void record_event(gbfft_plan_s* p, cudaStream_t stream, int pipe, bool first) {
  if (!p->time_stages) return;
  if (first) {
    gbfft_plan_s::TimedCall c;
    c.pipe = pipe;
    c.nev = 0;
    p->timed.push_back(c);
  }
  gbfft_plan_s::TimedCall& c = p->timed.back();
  if (c.nev > kMaxStages) return;
  if (cudaEventCreate(&c.ev[c.nev]) != cudaSuccess) return;
  cudaEventRecord(c.ev[c.nev], stream);
  ++c.nev;
}

static int run_persistent(gbfft_plan_s* p, const Pipeline& P, const PersistentKernel* pk, cudaStream_t stream,
                          unsigned warp_mask = 0, int tiles_per_ticket = 1);

// The fused plane kernel for stages s and s+1, if they are the two in-plane
// stages of a slab pipeline (stage s+1 reads only stage s's tiles of the same
// plane: rule kDepOuter over the same batch x outer planes) and one is built.
static const PlaneKernel* find_plane(const Pipeline& P, int s) {
  if (s + 1 >= P.n) return nullptr;
  const StageDesc& a = P.st[s];
  const StageDesc& b = P.st[s + 1];
  if (b.dep_rule != kDepOuter || a.batch != b.batch || a.n_outer != b.n_outer) return nullptr;
  if (a.prec != kPrecFP32 || b.prec != kPrecFP32 || a.n_tiles == 0 || b.n_tiles == 0) return nullptr;
  ensure_registry();
  for (const auto& k : plane_registry())
    if (k.L1 == a.L && k.dir1 == a.dir && k.kind1 == a.kind && k.L2 == b.L && k.dir2 == b.dir && k.kind2 == b.kind)
      return &k;
  return nullptr;
}

// The plane kernel with the intermediate in distributed shared memory for
// stages s and s+1: a real transform's in-plane pair (forward: the R2C x stage
// of 512-point rows, then y; inverse: y, then the C2R x stage) with contiguous
// rows, the y side in the natural spectrum layout, FP32, and a built length ny.
static const PlaneDsmKernel* find_plane_dsm(const Pipeline& P, int s) {
  if (s + 1 >= P.n) return nullptr;
  const StageDesc& a = P.st[s];
  const StageDesc& b = P.st[s + 1];
  if (b.dep_rule != kDepOuter || a.batch != b.batch || a.n_outer != b.n_outer || a.dir != b.dir) return nullptr;
  if (a.prec != kPrecFP32 || b.prec != kPrecFP32 || a.n_tiles == 0 || b.n_tiles == 0) return nullptr;
  if (a.m_split != 0 || b.m_split != 0) return nullptr;
  const bool fwd = a.dir < 0;
  const StageDesc& x = fwd ? a : b;
  const StageDesc& y = fwd ? b : a;
  if (x.kind != (fwd ? kR2CPost : kC2RPre) || x.L != kDsmM || y.kind != kPlain) return nullptr;
  if (!x.twn || !x.tw2 || !y.twn || x.n_group != y.L || y.n_group != kDsmM + 1) return nullptr;
  if (fwd) {
    if (x.in_mode != kRow || x.in_n != 1 || x.scale != 1.f) return nullptr;
    if (y.out_mode != kCol || y.out_g != 1 || y.out_n != kDsmM + 1) return nullptr;
  } else {
    if (x.out_mode != kRow || x.out_n != 1) return nullptr;
    if (y.in_mode != kCol || y.in_g != 1 || y.in_n != kDsmM + 1) return nullptr;
  }
  ensure_registry();
  for (const auto& k : plane_dsm_registry())
    if (k.ny == y.L && k.dir == a.dir) return &k;
  return nullptr;
}

// Bit s set for every stage s that starts a fusable in-plane pair.
static unsigned plane_mask_of(const Pipeline& P) {
  unsigned m = 0;
  for (int s = 0; s + 1 < P.n; ++s)
    if (find_plane(P, s) || find_plane_dsm(P, s)) {
      m |= 1u << s;
      ++s;
    }
  return m;
}

// One cluster per plane: `cx` CTAs (2, 4 or 8; 0 picks 8 for planes above
// 1.5 MB, as C2C 512^2, else 4), and no more CTAs than the larger stage has
// group chunks.
static int launch_plane(const PlaneKernel* k, const StageDesc& a, const StageDesc& b, cudaStream_t stream,
                        int cx = 0) {
  const long long plane_bytes = (long long)a.n_group * a.n_out * (long long)sizeof(float2);
  if (cx != 2 && cx != 4 && cx != 8) cx = plane_bytes > (3LL << 19) ? 8 : 4;
  while (cx > 1 && cx > std::max(a.n_gchunks, b.n_gchunks)) cx /= 2;
  const long long planes = (long long)a.batch * a.n_outer;
  if (planes * cx > 0x7FFFFFFFLL) return GBFFT_ERR_INVALID_ARG;
  int bpsm = 1;
  cudaError_t e = launch_info(k->fn, k->threads, k->smem, &bpsm);
  if (e != cudaSuccess) return GBFFT_ERR_CUDA;
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3((unsigned)(planes * cx));
  cfg.blockDim = dim3((unsigned)k->threads);
  cfg.dynamicSmemBytes = k->smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cx;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  StageDesc da = a, db = b;
  void* args[] = {&da, &db};
  return cuda_err(cudaLaunchKernelExC(&cfg, k->fn, args));
}

// Clusters of kDsmCta CTAs (one per SM: each holds 1/8 of a plane), as many as
// fit on the GPU at once, each running planes c, c + clusters, ...
static std::map<std::pair<int, const void*>, int> g_dsm_clusters;
static int launch_plane_dsm(const PlaneDsmKernel* k, const StageDesc& a, const StageDesc& b, cudaStream_t stream) {
  const long long planes = (long long)a.batch * a.n_outer;
  int bpsm = 1;
  cudaError_t e = launch_info(k->fn, k->threads, k->smem, &bpsm);
  if (e != cudaSuccess) return GBFFT_ERR_CUDA;
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.blockDim = dim3((unsigned)k->threads);
  cfg.dynamicSmemBytes = k->smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)kDsmCta;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GBFFT_ERR_CUDA;
  int clusters = 0;
  {
    std::lock_guard<std::mutex> lk(g_launch_mu);
    auto it = g_dsm_clusters.find({dev, k->fn});
    if (it != g_dsm_clusters.end()) {
      clusters = it->second;
    } else {
      cfg.gridDim = dim3((unsigned)kDsmCta);
      if (cudaOccupancyMaxActiveClusters(&clusters, k->fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return GBFFT_ERR_CUDA;
      }
      g_dsm_clusters[{dev, k->fn}] = clusters;
    }
  }
  if (clusters < 1) return GBFFT_ERR_UNSUPPORTED_SIZE;
  cfg.gridDim = dim3((unsigned)(std::min<long long>(planes, clusters) * kDsmCta));
  StageDesc da = a, db = b;
  void* args[] = {&da, &db};
  return cuda_err(cudaLaunchKernelExC(&cfg, k->fn, args));
}

// Staged launches with an explicit per-stage kernel choice (bit s of tma_mask:
// tensor-copy kernel for stage s when it can run there; bit s of plane_mask:
// stages s and s+1 as one fused plane launch when they form an in-plane pair).
static int run_staged(gbfft_plan_s* p, const Pipeline& P, unsigned tma_mask, cudaStream_t stream, int pipe,
                      unsigned plane_mask = 0, int plane_cx = 0, unsigned warp_mask = 0, unsigned prefetch_mask = 0,
                      bool plane_dsm = false) {
  record_event(p, stream, pipe, true);
  for (int s = 0; s < P.n; ++s) {
    if ((plane_mask >> s) & 1u) {
      const PlaneDsmKernel* kd = plane_dsm ? find_plane_dsm(P, s) : nullptr;
      if (kd) {
        int rc = launch_plane_dsm(kd, P.st[s], P.st[s + 1], stream);
        if (rc) return rc;
        record_event(p, stream, pipe, false);
        ++s;
        continue;
      }
      if (const PlaneKernel* k = find_plane(P, s)) {
        int rc = launch_plane(k, P.st[s], P.st[s + 1], stream, plane_cx);
        if (rc) return rc;
        record_event(p, stream, pipe, false);
        ++s;
        continue;
      }
    }
    const unsigned f = stage_flags((tma_mask >> s) & 1u, (warp_mask >> s) & 1u, (prefetch_mask >> s) & 1u);
    int rc = launch_stage(P.st[s], stream, f, &p->ctl->error);
    if (rc) return rc;
    record_event(p, stream, pipe, false);
  }
  return GBFFT_OK;
}

static int run_pipeline(gbfft_plan_s* p, const Pipeline& P, int pipe, cudaStream_t stream) {
  int vrc = validate(P);
  if (vrc) return vrc;
  if (p->tune[pipe].tuned) {
    const PersistentKernel* pk = p->tune[pipe].persistent ? find_persistent(P) : nullptr;
    if (pk) {
      record_event(p, stream, pipe, true);
      int rc = run_persistent(p, P, pk, stream, p->tune[pipe].warp_mask, p->tune[pipe].persistent_tiles);
      record_event(p, stream, pipe, false);
      return rc;
    }
    const gbfft_plan_s::Tuning& t = p->tune[pipe];
    return run_staged(p, P, t.tma_mask, stream, pipe, t.plane_mask, t.plane_cx, t.warp_mask, t.prefetch_mask,
                      t.plane_dsm);
  }
  const bool staged = (p->flags & GBFFT_STAGED) != 0;
  const unsigned tm = (p->flags & GBFFT_NO_TMA) ? 0u : 0xFFu;
  // slab pipelines: the in-plane stage pairs as fused plane launches unless staged
  const unsigned pm = (!staged && is_slab(p)) ? plane_mask_of(P) : 0u;
  if (pm) return run_staged(p, P, tm, stream, pipe, pm);
  const PersistentKernel* pk = staged ? nullptr : find_persistent(P);
  if (!pk) return run_staged(p, P, tm, stream, pipe);
  record_event(p, stream, pipe, true);
  int rc = run_persistent(p, P, pk, stream);
  record_event(p, stream, pipe, false);
  return rc;
}

// Stages of a persistent launch that can run the warp-per-pencil body (bit s).
static unsigned persistent_warp_mask(const Pipeline& P, const PersistentKernel* pk) {
  unsigned m = 0;
  if (!pk || !pk->warp_body) return 0;
  for (int s = 0; s < P.n; ++s)
    if (persistent_warp_body(pk->threads, P.st[s].L, P.st[s].kind) && P.st[s].twn && P.st[s].prec == kPrecFP32)
      m |= 1u << s;
  return m;
}

// warp_mask bit s: stage s runs the warp-per-pencil tile body (where it can).
// Write-after-read / write-after-write ordering inside one launch. The
// dependency rules order each tile after the producer tiles it reads, not
// after the tiles of earlier stages that read or wrote the buffer it
// overwrites (a pencil pipeline's last stage writes the output buffer that the
// middle stage reads and the first stage wrote). Stage s therefore waits for
// the whole of the latest earlier stage r that touched its output buffer,
// except the previous stage writing it for an in-place stage s (then s reads
// exactly what its producers wrote). The completion of stage r implies that of
// every stage before it: each tile of a stage is read by some tile of the next.
static void persistent_war(const Pipeline& P, int* war) {
  for (int s = 0; s < kMaxStages; ++s) war[s] = -1;
  for (int s = 1; s < P.n; ++s) {
    const void* o = P.st[s].out;
    for (int r = 0; r < s; ++r) {
      const bool reads = P.st[r].in == o, writes = P.st[r].out == o;
      if (r == s - 1 && !reads) continue;  // the producer writing what s reads (or nothing of o)
      if (reads || writes) war[s] = r;
    }
  }
}

static int run_persistent(gbfft_plan_s* p, const Pipeline& P, const PersistentKernel* pk, cudaStream_t stream,
                          unsigned warp_mask, int tiles_per_ticket) {
  PersistentArgs a;
  std::memset(&a, 0, sizeof(a));
  a.nstages = P.n;
  if (tiles_per_ticket != 1 && tiles_per_ticket != 2 && tiles_per_ticket != 4) return GBFFT_ERR_INVALID_ARG;
  a.tiles_per_ticket = tiles_per_ticket;
  const unsigned wm = warp_mask & persistent_warp_mask(P, pk);
  for (int s = 0; s < P.n; ++s) {
    a.st[s] = P.st[s];
    a.st[s].body = (wm >> s) & 1u;
  }
  long long total = 0;
  for (int s = 0; s < P.n; ++s) total += (P.st[s].n_tiles + tiles_per_ticket - 1) / tiles_per_ticket;
  if (total >= (1LL << 31)) return GBFFT_ERR_INVALID_ARG;
  a.total = (unsigned int)total;
  a.ctl = p->ctl;
  unsigned int* c = p->counters;
  for (int s = 0; s < P.n; ++s) {
    const StageDesc& d = P.st[s];
    a.cnt_outer[s] = c;
    c += (size_t)d.batch * d.n_outer;
    a.cnt_outer16[s] = c;
    c += (size_t)d.batch * gchunks(d.n_outer);
    a.cnt_gchunk[s] = c;
    c += (size_t)d.batch * d.n_gchunks;
    a.cnt_total[s] = c;
    c += (size_t)d.batch;
    a.cnt_stage[s] = c;
    c += 1;
  }
  const bool dbg = (p->flags & GBFFT_DEBUG_TIMEOUT) != 0;
  a.timeout_ns = dbg ? 20000000LL : 2000000000LL;
  a.debug_never = dbg ? 1 : 0;
  for (int s = 0; s < P.n; ++s) a.sig[s] = s + 1 < P.n ? persistent_sig_for_rule(P.st[s + 1].dep_rule) : 0;
  persistent_war(P, a.war);
  cudaError_t e = cudaMemsetAsync(&p->ctl->ticket, 0, 2 * sizeof(unsigned int) + p->counters_words * sizeof(unsigned int),
                                  stream);
  if (e != cudaSuccess) return GBFFT_ERR_CUDA;
  const size_t smem = pk->smem + (size_t)P.n * pk->tw_smem_per_stage;
  int bpsm = 1;
  e = launch_info(pk->fn, pk->threads, smem, &bpsm);
  if (e != cudaSuccess) return GBFFT_ERR_CUDA;
  long long grid = std::min<long long>((long long)a.total, (long long)sm_count() * bpsm);
  void* args[] = {&a};
  e = cudaLaunchKernel(pk->fn, dim3((unsigned)std::max<long long>(grid, 1)), dim3((unsigned)pk->threads), args,
                       smem, stream);
  return cuda_err(e);
}

static float2* upload_table(const std::vector<float2>& h) {
  float2* d = nullptr;
  if (cudaMalloc(&d, h.size() * sizeof(float2)) != cudaSuccess) return nullptr;
  if (cudaMemcpy(d, h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(d);
    return nullptr;
  }
  return d;
}

// W_n^t = exp(-2 pi i t / n) for t in [0, count), computed in FP64 and rounded once.
static std::vector<float2> twiddle_table(int n, int count) {
  std::vector<float2> h((size_t)count);
  const double two_pi = 6.283185307179586476925286766559;
  for (int t = 0; t < count; ++t) {
    double a = two_pi * ((double)(t % n) / (double)n);
    h[(size_t)t] = make_float2((float)std::cos(a), (float)-std::sin(a));
  }
  return h;
}

namespace gbfft {
// Packed Stockham twiddles of length L (the device layout of tw_table_len):
// pass i >= 1 with prefix Ns and radix R stores W_{Ns R}^{r k} at k R + r.
// Each value is exp(-2 pi i r k / (Ns R)) in FP64, rounded once to FP32.
std::vector<float2> packed_twiddles(int L) {
  int rad[16];
  const int np = host_radices(L, rad, 16);
  std::vector<float2> h;
  const double two_pi = 6.283185307179586476925286766559;
  long long ns = np > 0 ? rad[0] : 1;
  for (int i = 1; i < np; ++i) {
    const int R = rad[i];
    const long long m = ns * R;
    for (long long k = 0; k < ns; ++k)
      for (int r = 0; r < R; ++r) {
        double a = two_pi * ((double)((r * k) % m) / (double)m);
        h.push_back(make_float2((float)std::cos(a), (float)-std::sin(a)));
      }
    ns = m;
  }
  if (h.empty()) h.push_back(make_float2(1.f, 0.f));
  return h;
}
}  // namespace gbfft

static void free_plan(gbfft_plan_s* p) {
  if (!p) return;
  cudaFree(p->tw_x);
  cudaFree(p->tw_y);
  cudaFree(p->tw_z);
  cudaFree(p->tw2);
  if (p->ws_owned) cudaFree(p->ws);
  cudaFree(p->ctl);
  cudaFree(p->h_in_dev);
  cudaFree(p->h_out_dev);
  cudaFree(p->twn_x);
  cudaFree(p->twn_y);
  cudaFree(p->twn_z);
  cudaFree(p->twn_real);
  cudaFree(p->tw4_x);
  cudaFree(p->tw4_y);
  cudaFree(p->tw4_z);
  if (p->h_stream) cudaStreamDestroy(p->h_stream);
  if (p->h_stream2) cudaStreamDestroy(p->h_stream2);
  for (cudaEvent_t e : p->h_ev)
    if (e) cudaEventDestroy(e);
  for (auto& c : p->timed)
    for (int k = 0; k < c.nev; ++k) cudaEventDestroy(c.ev[k]);
  delete p;
}

// ------------------------------------------------------------------- C ABI

extern "C" {

const char* gbfft_version(void) { return "gbfft 0.1 (sm_103a)"; }

const char* gbfft_strerror(int code) {
  switch (code) {
    case GBFFT_OK:
      return "ok";
    case GBFFT_ERR_INVALID_ARG:
      return "invalid argument";
    case GBFFT_ERR_UNSUPPORTED_SIZE:
      return "unsupported transform length";
    case GBFFT_ERR_ALIGNMENT:
      return "pointer not 16-byte aligned";
    case GBFFT_ERR_INPLACE:
      return "in-place execution is not supported (in == out)";
    case GBFFT_ERR_ALLOC:
      return "device allocation failed or workspace too small";
    case GBFFT_ERR_CUDA:
      return "CUDA runtime error";
    case GBFFT_ERR_TIMEOUT:
      return "device dependency wait timed out";
    case GBFFT_ERR_NO_DEVICE:
      return "no CUDA device";
    case GBFFT_ERR_STATIC_LIMIT:
      return "grid larger than the static scratch of gbfft_exec_c2c_noalloc";
    case GBFFT_ERR_SETUP_IN_CAPTURE:
      return "gbfft_exec_c2c_noalloc: first call on this device made while its stream was capturing";
    default:
      return "unknown error";
  }
}

int gbfft_radix_plan(int n, int* radices, int cap) {
  if (!radices || cap < 0) return GBFFT_ERR_INVALID_ARG;
  int r = host_radices(n, radices, cap);
  return r < 0 ? GBFFT_ERR_UNSUPPORTED_SIZE : r;
}

int gbfft_supported_length(int n) { return (n >= 2 && stage_supported(n)) ? 1 : 0; }

int gbfft_workspace_size(gbfft_plan plan, size_t* bytes) {
  if (!plan || !bytes) return GBFFT_ERR_INVALID_ARG;
  *bytes = (size_t)plan->n_ws * spectrum_bytes(plan);
  return GBFFT_OK;
}

int gbfft_set_workspace(gbfft_plan plan, void* dev_ptr, size_t bytes) {
  if (!plan) return GBFFT_ERR_INVALID_ARG;
  size_t need = 0;
  gbfft_workspace_size(plan, &need);
  if (need == 0) return GBFFT_OK;
  if (!dev_ptr) return GBFFT_ERR_INVALID_ARG;
  if (((uintptr_t)dev_ptr) % 256 != 0) return GBFFT_ERR_ALIGNMENT;
  if (bytes < need) return GBFFT_ERR_ALLOC;
  if (plan->ws_owned) cudaFree(plan->ws);
  plan->ws = dev_ptr;
  plan->ws_bytes = bytes;
  plan->ws_owned = false;
  return GBFFT_OK;
}

int gbfft_plan_create(gbfft_plan* out, int nx, int ny, int nz, int kind, int dtype, int batch, unsigned flags) {
  if (!out) return GBFFT_ERR_INVALID_ARG;
  *out = nullptr;
  if (nx < 2 || ny < 2 || nz < 2 || batch < 1) return GBFFT_ERR_INVALID_ARG;
  if (kind != GBFFT_C2C && kind != GBFFT_R2C) return GBFFT_ERR_INVALID_ARG;
  if (dtype != GBFFT_FP32 && dtype != GBFFT_FP16_SPLIT && dtype != GBFFT_BF16_SPLIT && dtype != GBFFT_FP16_SPLIT_TC5 &&
      dtype != GBFFT_BF16_SPLIT_TC5)
    return GBFFT_ERR_INVALID_ARG;
  // split precision applies to the complex (kPlain) stages; the real x stage of R2C plans and the
  // fused Poisson z stages keep FP32
  const unsigned known = GBFFT_SLAB | GBFFT_TRANSPOSED_OUT | GBFFT_STAGED | GBFFT_NO_TMA | GBFFT_DEBUG_TIMEOUT;
  if (flags & ~known) return GBFFT_ERR_INVALID_ARG;
  if ((flags & GBFFT_SLAB) && (flags & GBFFT_TRANSPOSED_OUT)) return GBFFT_ERR_INVALID_ARG;
  if (kind == GBFFT_R2C && (nx % 2 != 0 || nx < 4)) return GBFFT_ERR_INVALID_ARG;
  const int Lx = kind == GBFFT_R2C ? nx / 2 : nx;
  if (!stage_supported(Lx) || !stage_supported(ny) || !stage_supported(nz)) return GBFFT_ERR_UNSUPPORTED_SIZE;
  for (int L : {kind == GBFFT_R2C ? ny : nx, ny, nz})
    if (dtype != GBFFT_FP32 && (!find_stage(L, -1, kPlain, dtype) || !find_stage(L, 1, kPlain, dtype)))
      return GBFFT_ERR_UNSUPPORTED_SIZE;
  if (kind == GBFFT_R2C && (!find_stage(Lx, -1, kR2CPost) || !find_stage(Lx, 1, kC2RPre)))
    return GBFFT_ERR_UNSUPPORTED_SIZE;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return GBFFT_ERR_NO_DEVICE;
  }
  gbfft_plan_s* p = new gbfft_plan_s();
  p->nx = nx;
  p->ny = ny;
  p->nz = nz;
  p->batch = batch;
  p->kind = kind;
  p->dtype = dtype;
  p->flags = flags;
  cudaGetDevice(&p->device);
  p->nxc = kind == GBFFT_R2C ? nx / 2 + 1 : nx;
  p->Lx = Lx;
  p->rowA = Lx;  // complex values per input row (real pairs for R2C)
  p->Nc = (long long)p->nxc * ny * nz;
  p->NA = (long long)p->rowA * ny * nz;
  // tickets of a persistent launch are 32-bit
  if ((long long)batch * std::max<long long>((long long)nz * gchunks(ny),
                                             std::max<long long>((long long)p->nxc * gchunks(nz),
                                                                 (long long)ny * gchunks(p->nxc))) >=
      (1LL << 29)) {
    delete p;
    return GBFFT_ERR_INVALID_ARG;
  }
  // workspace buffers: pencil C2C 1; pencil R2C 2 (inverse, Poisson); slab R2C 1; slab C2C 0
  if (!is_slab(p))
    p->n_ws = kind == GBFFT_R2C ? 2 : 1;
  else
    p->n_ws = kind == GBFFT_R2C ? 1 : 0;

  p->tw_x = upload_table(packed_twiddles(Lx));
  p->tw_y = upload_table(packed_twiddles(ny));
  p->tw_z = upload_table(packed_twiddles(nz));
  p->twn_x = upload_table(twiddle_table(Lx, Lx));
  p->twn_y = upload_table(twiddle_table(ny, ny));
  p->twn_z = upload_table(twiddle_table(nz, nz));
  bool ok = p->tw_x && p->tw_y && p->tw_z && p->twn_x && p->twn_y && p->twn_z;
  if (ok) {
    p->tw4_x = upload_table(twiddle_table(4 * Lx, Lx + 1));
    p->tw4_y = upload_table(twiddle_table(4 * ny, ny + 1));
    p->tw4_z = upload_table(twiddle_table(4 * nz, nz + 1));
    ok = p->tw4_x && p->tw4_y && p->tw4_z;
  }
  if (ok && kind == GBFFT_R2C) {
    p->tw2 = upload_table(twiddle_table(2 * Lx, Lx + 1));
    p->twn_real = upload_table(twiddle_table(nx, nx));
    ok = p->tw2 != nullptr && p->twn_real != nullptr;
  }
  // persistent-launch counters: sized for the largest pipeline
  size_t words = 0;
  for (int pipe = 0; pipe < kNumPipes && ok; ++pipe) {
    if (pipe == kPipePoisson && kind != GBFFT_R2C) continue;
    int op = pipe == kPipeFwd ? GBFFT_OP_FORWARD : (pipe == kPipeInv ? GBFFT_OP_INVERSE : 4);
    const Buf none{nullptr, -1};
    Pipeline P = build_pipeline(p, pipe, op, none, none, none, none);
    words = std::max(words, counter_words(P));
  }
  if (ok) {
    p->counters_words = words;
    void* c = nullptr;
    if (cudaMalloc(&c, sizeof(Control) + words * sizeof(unsigned int)) != cudaSuccess) {
      ok = false;
    } else {
      p->ctl = reinterpret_cast<Control*>(c);
      p->counters = reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(c) + sizeof(Control));
      ok = cudaMemset(c, 0, sizeof(Control) + words * sizeof(unsigned int)) == cudaSuccess;
    }
  }
  if (!ok) {
    cudaGetLastError();
    free_plan(p);
    return GBFFT_ERR_ALLOC;
  }
  *out = p;
  return GBFFT_OK;
}

void gbfft_plan_destroy(gbfft_plan plan) { free_plan(plan); }

static int check_ptrs(const void* in, const void* out) {
  if (!in || !out) return GBFFT_ERR_INVALID_ARG;
  if (in == out) return GBFFT_ERR_INPLACE;
  if (((uintptr_t)in) % 16 != 0 || ((uintptr_t)out) % 16 != 0) return GBFFT_ERR_ALIGNMENT;
  return GBFFT_OK;
}

static Buf ws_buf(gbfft_plan_s* p, int i) {
  if (!p->ws || i >= p->n_ws) return Buf{nullptr, 0};
  return Buf{reinterpret_cast<char*>(p->ws) + (size_t)i * spectrum_bytes(p),
             (long long)(spectrum_bytes(p) / sizeof(float2))};
}

static size_t op_in_bytes(const gbfft_plan_s* p, int op);
static size_t op_out_bytes(const gbfft_plan_s* p, int op);

int gbfft_exec(gbfft_plan plan, int op, const void* in, void* out, void* stream) {
  if (!plan) return GBFFT_ERR_INVALID_ARG;
  if (op < GBFFT_OP_FORWARD || op > GBFFT_OP_INVERSE_ADJOINT) return GBFFT_ERR_INVALID_ARG;
  int rc = check_ptrs(in, out);
  if (rc) return rc;
  if (cudaSetDevice(plan->device) != cudaSuccess) return GBFFT_ERR_CUDA;
  rc = ensure_workspace(plan);
  if (rc) return rc;
  const int pipe = pipe_of(op);
  Buf bin{const_cast<void*>(in), (long long)(op_in_bytes(plan, op) / sizeof(float2))};
  Buf bout{out, (long long)(op_out_bytes(plan, op) / sizeof(float2))};
  Pipeline P = build_pipeline(plan, pipe, op, bin, bout, ws_buf(plan, 0), ws_buf(plan, 1));
  return run_pipeline(plan, P, pipe, reinterpret_cast<cudaStream_t>(stream));
}

int gbfft_exec_forward(gbfft_plan plan, const void* in, void* out, void* stream) {
  return gbfft_exec(plan, GBFFT_OP_FORWARD, in, out, stream);
}
int gbfft_exec_inverse(gbfft_plan plan, const void* in, void* out, void* stream) {
  return gbfft_exec(plan, GBFFT_OP_INVERSE, in, out, stream);
}
int gbfft_exec_adjoint(gbfft_plan plan, const void* in, void* out, void* stream) {
  return gbfft_exec(plan, GBFFT_OP_ADJOINT, in, out, stream);
}
int gbfft_exec_inverse_adjoint(gbfft_plan plan, const void* in, void* out, void* stream) {
  return gbfft_exec(plan, GBFFT_OP_INVERSE_ADJOINT, in, out, stream);
}

}  // extern "C"

// op 4: periodic z; op 5: bounded z (DCT)
static int exec_poisson_op(gbfft_plan plan, int op, const void* in, void* out, void* stream) {
  if (!plan) return GBFFT_ERR_INVALID_ARG;
  if (plan->kind != GBFFT_R2C || plan->batch < 1) return GBFFT_ERR_INVALID_ARG;
  if (!find_stage(plan->nz, -1, op == 5 ? kPoissonZB : kPoissonZ)) return GBFFT_ERR_UNSUPPORTED_SIZE;
  int rc = check_ptrs(in, out);
  if (rc) return rc;
  if (cudaSetDevice(plan->device) != cudaSuccess) return GBFFT_ERR_CUDA;
  rc = ensure_workspace(plan);
  if (rc) return rc;
  Buf bin{const_cast<void*>(in), (long long)(op_in_bytes(plan, op) / sizeof(float2))};
  Buf bout{out, (long long)(op_out_bytes(plan, op) / sizeof(float2))};
  Pipeline P = build_pipeline(plan, kPipePoisson, op, bin, bout, ws_buf(plan, 0), ws_buf(plan, 1));
  return run_pipeline(plan, P, kPipePoisson, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" {

int gbfft_exec_poisson(gbfft_plan plan, const void* in, void* out, void* stream) {
  return exec_poisson_op(plan, 4, in, out, stream);
}

int gbfft_exec_poisson_bounded(gbfft_plan plan, const void* in, void* out, void* stream) {
  return exec_poisson_op(plan, 5, in, out, stream);
}

int gbfft_exec_r2r(gbfft_plan plan, int r2r_x, int r2r_y, int r2r_z, int inverse, const void* in, void* out,
                   void* stream) {
  if (!plan || (inverse != 0 && inverse != 1)) return GBFFT_ERR_INVALID_ARG;
  const int r2r[3] = {r2r_x, r2r_y, r2r_z};
  const int len[3] = {plan->nx, plan->ny, plan->nz};
  for (int ax = 0; ax < 3; ++ax) {
    if (r2r[ax] != GBFFT_R2R_NONE && r2r[ax] != GBFFT_R2R_DCT && r2r[ax] != GBFFT_R2R_DST)
      return GBFFT_ERR_INVALID_ARG;
    if (r2r[ax] == GBFFT_R2R_NONE) continue;
    if (ax == 0 && plan->kind == GBFFT_R2C) return GBFFT_ERR_INVALID_ARG;  // x of an R2C plan is the real axis
    const bool dct = r2r[ax] == GBFFT_R2R_DCT;
    const int kind = inverse ? (dct ? kDct3 : kDst3) : (dct ? kDct2 : kDst2);
    if (!find_stage(len[ax], inverse ? 1 : -1, kind)) return GBFFT_ERR_UNSUPPORTED_SIZE;
  }
  int rc = check_ptrs(in, out);
  if (rc) return rc;
  if (cudaSetDevice(plan->device) != cudaSuccess) return GBFFT_ERR_CUDA;
  rc = ensure_workspace(plan);
  if (rc) return rc;
  const int op = inverse ? GBFFT_OP_INVERSE : GBFFT_OP_FORWARD;
  const int pipe = pipe_of(op);
  Buf bin{const_cast<void*>(in), (long long)(op_in_bytes(plan, op) / sizeof(float2))};
  Buf bout{out, (long long)(op_out_bytes(plan, op) / sizeof(float2))};
  Pipeline P = build_pipeline(plan, pipe, op, bin, bout, ws_buf(plan, 0), ws_buf(plan, 1), r2r);
  return run_pipeline(plan, P, pipe, reinterpret_cast<cudaStream_t>(stream));
}

int gbfft_exec_r2r_z(gbfft_plan plan, int r2r, int inverse, const void* in, void* out, void* stream) {
  if (r2r != GBFFT_R2R_DCT && r2r != GBFFT_R2R_DST) return GBFFT_ERR_INVALID_ARG;
  return gbfft_exec_r2r(plan, GBFFT_R2R_NONE, GBFFT_R2R_NONE, r2r, inverse, in, out, stream);
}

static size_t op_in_bytes(const gbfft_plan_s* p, int op) {
  const size_t real_b = (size_t)p->NA * p->batch * sizeof(float2);  // rowA complex per row
  const size_t spec_b = (size_t)p->Nc * p->batch * sizeof(float2);
  if (p->kind == GBFFT_C2C) return spec_b;
  if (op == GBFFT_OP_FORWARD || op == GBFFT_OP_INVERSE_ADJOINT || op == 4 || op == 5) return real_b;
  return spec_b;
}

static size_t op_out_bytes(const gbfft_plan_s* p, int op) {
  const size_t real_b = (size_t)p->NA * p->batch * sizeof(float2);
  const size_t spec_b = (size_t)p->Nc * p->batch * sizeof(float2);
  if (p->kind == GBFFT_C2C) return spec_b;
  if (op == GBFFT_OP_FORWARD || op == GBFFT_OP_INVERSE_ADJOINT) return spec_b;
  return real_b;
}

// The part of stage d's array on one side for outer indices [o0, o1) of a
// one-batch stage, as a 2D region of `rows` rows of `width` bytes at `pitch`
// (element offset `off`); false if the outer blocks are not contiguous there.
static bool outer_region(long long o_stride, long long g_stride, long long n_stride, int n_group, int n_len,
                         int mode, long long o0, long long o1, long long* off, size_t* width, size_t* pitch,
                         size_t* rows) {
  if ((long long)n_group * g_stride != o_stride) return false;
  if (mode == kRow) {
    if (n_stride != 1) return false;
    *off = o0 * o_stride;
    *width = (size_t)((o1 - o0) * o_stride) * sizeof(float2);
    *pitch = *width;
    *rows = 1;
    return true;
  }
  if (g_stride != 1) return false;
  *off = o0 * o_stride;
  *width = (size_t)((o1 - o0) * o_stride) * sizeof(float2);
  *pitch = (size_t)n_stride * sizeof(float2);
  *rows = (size_t)n_len;
  return true;
}

static cudaError_t copy_region(void* dst, const void* src, long long off, size_t width, size_t pitch, size_t rows,
                               cudaMemcpyKind kind, cudaStream_t s) {
  const char* sp = reinterpret_cast<const char*>(src) + off * (long long)sizeof(float2);
  char* dp = reinterpret_cast<char*>(dst) + off * (long long)sizeof(float2);
  if (rows == 1 || width == pitch) return cudaMemcpyAsync(dp, sp, width * rows, kind, s);
  return cudaMemcpy2DAsync(dp, pitch, sp, pitch, width, rows, kind, s);
}

// Host-buffer execution with the copies overlapped with the first and last
// stages: a first stage that reads rows runs on K slabs of its outer axis,
// each after its slab's host-to-device copy; a last stage that writes rows
// runs on K slabs, and each slab's device-to-host copy starts as soon as the
// slab is written (the column sides, whose slabs would be strided, move in
// one copy). Pencil plans
// with natural output, one batch entry, ops 0-3; the stages run as staged
// launches with the plan's tuned per-stage kernels. Returns 1 when the plan
// or op does not qualify (the caller takes the plain path).
static int exec_host_chunked(gbfft_plan_s* p, int op, const void* hin, void* hout, int K) {
  if (is_slab(p) || (p->flags & GBFFT_TRANSPOSED_OUT) || p->batch != 1 || op < 0 || op > 3) return 1;
  const int pipe = pipe_of(op);
  const long long cap_in = (long long)(p->h_in_bytes / sizeof(float2));
  int rc = ensure_workspace(p);
  if (rc) return rc;
  Pipeline P = build_pipeline(p, pipe, op, Buf{p->h_in_dev, cap_in}, Buf{p->h_out_dev, cap_in}, ws_buf(p, 0),
                              ws_buf(p, 1));
  if (P.n != 3) return 1;
  rc = validate(P);
  if (rc) return rc;
  const StageDesc& a = P.st[0];
  const StageDesc& z = P.st[2];
  if (a.batch != 1 || z.batch != 1) return 1;
  // the per-stage kernel choice of the plan's tuning (staged), else the staged defaults
  const gbfft_plan_s::Tuning& t = p->tune[pipe];
  const bool use_t = t.tuned && !t.persistent && !t.plane_mask;
  unsigned f[3];
  for (int s = 0; s < 3; ++s) {
    const bool tma = use_t ? ((t.tma_mask >> s) & 1u) : !(p->flags & GBFFT_NO_TMA);
    f[s] = stage_flags(tma, use_t && ((t.warp_mask >> s) & 1u), use_t && ((t.prefetch_mask >> s) & 1u));
  }
  // slabs only where they are contiguous (the row side: the real or natural rows of the x stage); a
  // column side (the natural spectrum of the z stage) moves in one copy -- its slabs would be strided 2D
  // copies, measured slower than one contiguous copy
  const int ka = a.in_mode == kRow ? std::min<int>(K, a.n_outer) : 1;
  const int kz = z.out_mode == kRow ? std::min<int>(K, z.n_outer) : 1;
  long long off;
  size_t w, pitch, rows;
  // the slabs of the first stage's input and the last stage's output must be contiguous or 2D regions
  if (!outer_region(a.in_o, a.in_g, a.in_n, a.n_group, a.n_in, a.in_mode, 0, 1, &off, &w, &pitch, &rows) ||
      !outer_region(z.out_o, z.out_g, z.out_n, z.n_group, z.n_out, z.out_mode, 0, 1, &off, &w, &pitch, &rows))
    return 1;
  if (!p->h_stream2 && cudaStreamCreateWithFlags(&p->h_stream2, cudaStreamNonBlocking) != cudaSuccess)
    return GBFFT_ERR_CUDA;
  for (cudaEvent_t& e : p->h_ev)
    if (!e && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return GBFFT_ERR_CUDA;
  cudaStream_t cs = p->h_stream, ks = p->h_stream2;
  int* err = &p->ctl->error;
  // first stage: slab k after its copy
  for (int k = 0; k < ka; ++k) {
    const long long o0 = (long long)a.n_outer * k / ka, o1 = (long long)a.n_outer * (k + 1) / ka;
    outer_region(a.in_o, a.in_g, a.in_n, a.n_group, a.n_in, a.in_mode, o0, o1, &off, &w, &pitch, &rows);
    if (copy_region(p->h_in_dev, hin, off, w, pitch, rows, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaEventRecord(p->h_ev[k], cs) != cudaSuccess || cudaStreamWaitEvent(ks, p->h_ev[k], 0) != cudaSuccess)
      return GBFFT_ERR_CUDA;
    StageDesc d = a;
    d.in += o0 * a.in_o;
    d.out += o0 * a.out_o;
    d.n_outer = (int)(o1 - o0);
    d.n_tiles = (long long)d.n_outer * d.n_gchunks;
    rc = launch_stage(d, ks, f[0], err);
    if (rc) return rc;
  }
  rc = launch_stage(P.st[1], ks, f[1], err);
  if (rc) return rc;
  // last stage: slab k, then its copy
  for (int k = 0; k < kz; ++k) {
    const long long o0 = (long long)z.n_outer * k / kz, o1 = (long long)z.n_outer * (k + 1) / kz;
    StageDesc d = z;
    d.in += o0 * z.in_o;
    d.out += o0 * z.out_o;
    d.n_outer = (int)(o1 - o0);
    d.n_tiles = (long long)d.n_outer * d.n_gchunks;
    rc = launch_stage(d, ks, f[2], err);
    if (rc) return rc;
    outer_region(z.out_o, z.out_g, z.out_n, z.n_group, z.n_out, z.out_mode, o0, o1, &off, &w, &pitch, &rows);
    if (cudaEventRecord(p->h_ev[16 + k], ks) != cudaSuccess || cudaStreamWaitEvent(cs, p->h_ev[16 + k], 0) != cudaSuccess ||
        copy_region(hout, p->h_out_dev, off, w, pitch, rows, cudaMemcpyDeviceToHost, cs) != cudaSuccess)
      return GBFFT_ERR_CUDA;
  }
  return cuda_err(cudaStreamSynchronize(cs));
}

int gbfft_plan_set_host_chunks(gbfft_plan plan, int chunks) {
  if (!plan || chunks < 1 || chunks > 16) return GBFFT_ERR_INVALID_ARG;
  plan->host_chunks = chunks;
  return GBFFT_OK;
}

int gbfft_exec_host(gbfft_plan plan, int op, const void* host_in, void* host_out) {
  if (!plan || !host_in || !host_out) return GBFFT_ERR_INVALID_ARG;
  if (op < 0 || op > 5) return GBFFT_ERR_INVALID_ARG;
  if (cudaSetDevice(plan->device) != cudaSuccess) return GBFFT_ERR_CUDA;
  const size_t ib = op_in_bytes(plan, op), ob = op_out_bytes(plan, op);
  if (!plan->h_stream && cudaStreamCreateWithFlags(&plan->h_stream, cudaStreamNonBlocking) != cudaSuccess)
    return GBFFT_ERR_CUDA;
  const size_t big = std::max(op_in_bytes(plan, 0), op_out_bytes(plan, 0));
  if (!plan->h_in_dev) {
    if (cudaMalloc(&plan->h_in_dev, big) != cudaSuccess || cudaMalloc(&plan->h_out_dev, big) != cudaSuccess) {
      cudaGetLastError();
      return GBFFT_ERR_ALLOC;
    }
    plan->h_in_bytes = plan->h_out_bytes = big;
  }
  if (plan->host_chunks > 1) {
    const int crc = exec_host_chunked(plan, op, host_in, host_out, plan->host_chunks);
    if (crc != 1) return crc;
  }
  cudaStream_t s = plan->h_stream;
  if (cudaMemcpyAsync(plan->h_in_dev, host_in, ib, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return GBFFT_ERR_CUDA;
  int rc = op == 5   ? gbfft_exec_poisson_bounded(plan, plan->h_in_dev, plan->h_out_dev, s)
           : op == 4 ? gbfft_exec_poisson(plan, plan->h_in_dev, plan->h_out_dev, s)
                   : gbfft_exec(plan, op, plan->h_in_dev, plan->h_out_dev, s);
  if (rc) return rc;
  if (cudaMemcpyAsync(host_out, plan->h_out_dev, ob, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return GBFFT_ERR_CUDA;
  return cuda_err(cudaStreamSynchronize(s));
}

int gbfft_get_device_error(gbfft_plan plan, int* code) {
  if (!plan || !code) return GBFFT_ERR_INVALID_ARG;
  if (cudaSetDevice(plan->device) != cudaSuccess) return GBFFT_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return GBFFT_ERR_CUDA;
  Control c;
  if (cudaMemcpy(&c, plan->ctl, sizeof(Control), cudaMemcpyDeviceToHost) != cudaSuccess) return GBFFT_ERR_CUDA;
  *code = c.error == kDevErrTimeout ? GBFFT_ERR_TIMEOUT : (c.error ? GBFFT_ERR_CUDA : GBFFT_OK);
  if (cudaMemset(plan->ctl, 0, sizeof(Control)) != cudaSuccess) return GBFFT_ERR_CUDA;
  return GBFFT_OK;
}

int gbfft_debug_run(gbfft_plan plan, int step, const void* in, void* out, void* stream) {
  if (!plan) return GBFFT_ERR_INVALID_ARG;
  int rc = check_ptrs(in, out);
  if (rc) return rc;
  if (cudaSetDevice(plan->device) != cudaSuccess) return GBFFT_ERR_CUDA;
  const bool fwd = step >= 1 && step <= 6;
  const bool inv = step >= 11 && step <= 16;
  if (!fwd && !inv) return GBFFT_ERR_INVALID_ARG;
  const int local = fwd ? step : step - 10;
  const bool identity = (local % 2) == 0;
  const int which = (local - 1) / 2;  // forward: 0 x, 1 y, 2 z; inverse: 0 z, 1 y, 2 x
  if (identity && plan->kind == GBFFT_R2C && ((fwd && which == 0) || (inv && which == 2)))
    return GBFFT_ERR_INVALID_ARG;
  if (is_slab(plan)) return GBFFT_ERR_INVALID_ARG;
  // pencil stage descriptors; only the selected stage's buffers matter
  gbfft_plan_s tmp = *plan;
  tmp.flags &= ~GBFFT_TRANSPOSED_OUT;
  const Buf none{nullptr, -1};
  Pipeline P = build_pipeline(&tmp, fwd ? kPipeFwd : kPipeInv, fwd ? GBFFT_OP_FORWARD : GBFFT_OP_ADJOINT, none,
                              none, none, none);
  StageDesc d = P.st[which];
  d.in = reinterpret_cast<const float2*>(in);
  d.out = reinterpret_cast<float2*>(out);
  d.scale = 1.f;
  d.interior = 1.f;
  d.dep_rule = kDepNone;
  if (identity) d.kind = kIdentity, d.dir = -1, d.n_in = d.n_out = d.L;
  return launch_stage(d, reinterpret_cast<cudaStream_t>(stream), plan->flags, &plan->ctl->error);
}

}  // extern "C"

// ----------------------------------------------------------- autotuning

// Whether stage d can run with the tensor-copy kernel (one exists for its
// length/kind/side and its input layout has a tensor map).
static bool tma_possible(const StageDesc& d) {
  if (d.kind == kIdentity || d.prec != kPrecFP32) return false;
  const int src = d.in_mode == kRow ? 1 : 2;
  if (!find_tma(d.L, d.dir, d.kind, src)) return false;
  alignas(64) CUtensorMap m;
  return encode_input_map(d, src, &m);
}

// Average time of `reps` back-to-back calls of f on `stream` after one warm-up
// call (CUDA events on the launching stream). Negative on failure.
template <typename F>
static float time_calls(F f, cudaStream_t stream, int reps) {
  if (f() != GBFFT_OK) return -1.f;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1.f;
  }
  cudaEventRecord(e0, stream);
  bool ok = true;
  for (int i = 0; i < reps && ok; ++i) ok = f() == GBFFT_OK;
  cudaEventRecord(e1, stream);
  float ms = -1.f;
  if (ok && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
    ms /= (float)reps;
  else
    ms = -1.f;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms;
}

extern "C" {

int gbfft_plan_autotune(gbfft_plan plan, void* stream) {
  if (!plan) return GBFFT_ERR_INVALID_ARG;
  if (cudaSetDevice(plan->device) != cudaSuccess) return GBFFT_ERR_CUDA;
  int rc = ensure_workspace(plan);
  if (rc) return rc;
  const size_t big = std::max(op_in_bytes(plan, 0), op_out_bytes(plan, 0));
  if (!plan->h_in_dev) {
    if (cudaMalloc(&plan->h_in_dev, big) != cudaSuccess || cudaMalloc(&plan->h_out_dev, big) != cudaSuccess) {
      cudaGetLastError();
      return GBFFT_ERR_ALLOC;
    }
    plan->h_in_bytes = plan->h_out_bytes = big;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(plan->h_in_dev, 0, big, st) != cudaSuccess) return GBFFT_ERR_CUDA;
  const bool was_timing = plan->time_stages;
  plan->time_stages = false;
  const int npipes = plan->kind == GBFFT_R2C ? 3 : 2;
  const int reps = 5;
  for (int pipe = 0; pipe < npipes; ++pipe) {
    const int op = pipe == kPipeFwd ? GBFFT_OP_FORWARD : (pipe == kPipeInv ? GBFFT_OP_INVERSE : 4);
    Buf bin{plan->h_in_dev, (long long)(big / sizeof(float2))};
    Buf bout{plan->h_out_dev, (long long)(big / sizeof(float2))};
    Pipeline P = build_pipeline(plan, pipe, op, bin, bout, ws_buf(plan, 0), ws_buf(plan, 1));
    rc = validate(P);
    if (rc) return rc;
    gbfft_plan_s::Tuning t;
    float staged_ms = 0.f;
    for (int s = 0; s < P.n; ++s) {
      const StageDesc d = P.st[s];
      float best = time_calls([&] { return launch_stage(d, st, GBFFT_NO_TMA, &plan->ctl->error); }, st, reps);
      if (best < 0.f) return GBFFT_ERR_CUDA;
      if (!(plan->flags & GBFFT_NO_TMA) && tma_possible(d)) {
        float tt = time_calls([&] { return launch_stage(d, st, 0u, &plan->ctl->error); }, st, reps);
        if (tt >= 0.f && tt < best) {
          best = tt;
          t.tma_mask |= 1u << s;
        }
      }
      if (find_warp(d)) {
        float tw = time_calls([&] { return launch_stage(d, st, GBFFT_NO_TMA | kUseWarpKernel, &plan->ctl->error); },
                              st, reps);
        if (tw >= 0.f && tw < best) {
          best = tw;
          t.tma_mask &= ~(1u << s);
          t.warp_mask |= 1u << s;
        }
      }
      if (s < 4 && find_prefetch(d)) {
        float tq = time_calls(
            [&] { return launch_stage(d, st, GBFFT_NO_TMA | kUsePrefetchKernel, &plan->ctl->error); }, st, reps);
        if (tq >= 0.f && tq < best) {
          best = tq;
          t.tma_mask &= ~(1u << s);
          t.warp_mask &= ~(1u << s);
          t.prefetch_mask |= 1u << s;
        }
      }
      t.stage_ms[s] = best;
      staged_ms += best;
    }
    t.ms = staged_ms;
    // the staged choice; a persistent launch below replaces the masks by its own
    const unsigned tm = t.tma_mask, wm = t.warp_mask, qm = t.prefetch_mask;
    const PersistentKernel* pk = (plan->flags & GBFFT_STAGED) ? nullptr : find_persistent(P);
    if (pk) {
      // one launch per transform: Stockham tile bodies, then the warp-per-pencil body on its length-512
      // complex stages, each with 1, 2 or 4 tiles per ticket
      const unsigned pw = persistent_warp_mask(P, pk);
      for (unsigned wmask : {0u, pw}) {
        for (int tpt : {1, 2, 4}) {
          float tp = time_calls([&] { return run_persistent(plan, P, pk, st, wmask, tpt); }, st, reps);
          if (tp >= 0.f && tp < t.ms) {
            t.persistent = true;
            t.ms = tp;
            t.tma_mask = t.prefetch_mask = 0;
            t.warp_mask = wmask;
            t.persistent_tiles = tpt;
          }
        }
        if (pw == 0u) break;
      }
    }
    const unsigned pm = (plan->flags & GBFFT_STAGED) ? 0u : plane_mask_of(P);
    if (pm) {
      // cluster plane launches through L2 (2, 4 or 8 CTAs per plane), then with the intermediate in
      // distributed shared memory (cx = 0 marks that candidate)
      for (int cx : {2, 4, 8, 0}) {
        const bool dsm = cx == 0;
        if (dsm) {
          bool any = false;
          for (int s = 0; s + 1 < P.n; ++s) any = any || (((pm >> s) & 1u) && find_plane_dsm(P, s));
          if (!any) continue;
        }
        float tf = time_calls([&] { return run_staged(plan, P, tm, st, pipe, pm, cx, wm, qm, dsm); }, st, reps);
        if (tf >= 0.f && tf < t.ms) {
          t.persistent = false;
          t.plane_mask = pm;
          t.plane_cx = cx;
          t.plane_dsm = dsm;
          t.ms = tf;
          t.tma_mask = tm;
          t.warp_mask = wm;
          t.prefetch_mask = qm;
        }
      }
    }
    t.tuned = true;
    plan->tune[pipe] = t;
  }
  plan->time_stages = was_timing;
  return cuda_err(cudaStreamSynchronize(st));
}

int gbfft_plan_get_tuning(gbfft_plan plan, int pipeline, int* tuned, int* persistent, unsigned* tma_mask,
                          float* ms, float* stage_ms) {
  if (!plan || pipeline < 0 || pipeline > 2) return GBFFT_ERR_INVALID_ARG;
  const gbfft_plan_s::Tuning& t = plan->tune[pipeline];
  if (tuned) *tuned = t.tuned ? 1 : 0;
  if (persistent) *persistent = t.persistent ? 1 : 0;
  if (tma_mask)
    *tma_mask = (t.tma_mask & 0xFFu) | ((t.plane_mask & 0xFFu) << 8) | ((unsigned)(t.plane_cx & 0xF) << 16) |
                ((t.warp_mask & 0x1Fu) << 20) | ((unsigned)(t.persistent_tiles == 4 ? 2 : t.persistent_tiles == 2 ? 1 : 0) << 25) |
                ((t.plane_dsm ? 1u : 0u) << 27) | ((t.prefetch_mask & 0xFu) << 28);
  if (ms) *ms = t.ms;
  if (stage_ms)
    for (int s = 0; s < kMaxStages; ++s) stage_ms[s] = t.stage_ms[s];
  return GBFFT_OK;
}

int gbfft_plan_set_tuning(gbfft_plan plan, int pipeline, int persistent, unsigned tma_mask) {
  if (!plan || pipeline < 0 || pipeline > 2) return GBFFT_ERR_INVALID_ARG;
  if (((tma_mask >> 25) & 0x3u) == 3u) return GBFFT_ERR_INVALID_ARG;  // tiles per ticket 1, 2 or 4
  gbfft_plan_s::Tuning& t = plan->tune[pipeline];
  t.tuned = true;
  t.persistent = persistent != 0;
  t.tma_mask = tma_mask & 0xFFu;
  t.plane_mask = (tma_mask >> 8) & 0xFFu;
  t.plane_cx = (int)((tma_mask >> 16) & 0xFu);
  t.warp_mask = (tma_mask >> 20) & 0x1Fu;
  t.persistent_tiles = 1 << ((tma_mask >> 25) & 0x3u);
  t.prefetch_mask = (tma_mask >> 28) & 0xFu;
  t.plane_dsm = ((tma_mask >> 27) & 1u) != 0;
  t.ms = 0.f;
  for (int s = 0; s < kMaxStages; ++s) t.stage_ms[s] = 0.f;
  return GBFFT_OK;
}

int gbfft_plan_time_stages(gbfft_plan plan, int enable) {
  if (!plan) return GBFFT_ERR_INVALID_ARG;
  plan->time_stages = enable != 0;
  return GBFFT_OK;
}

int gbfft_plan_stage_times(gbfft_plan plan, int pipeline, float* avg_ms, int* nsegments, int* ncalls) {
  if (!plan || !avg_ms || !nsegments || !ncalls || pipeline < 0 || pipeline > 2) return GBFFT_ERR_INVALID_ARG;
  if (cudaSetDevice(plan->device) != cudaSuccess) return GBFFT_ERR_CUDA;
  for (int s = 0; s < kMaxStages; ++s) avg_ms[s] = 0.f;
  *nsegments = 0;
  *ncalls = 0;
  std::vector<gbfft_plan_s::TimedCall> keep;
  for (auto& c : plan->timed) {
    if (c.pipe != pipeline) {
      keep.push_back(c);
      continue;
    }
    if (c.nev >= 2 && cudaEventSynchronize(c.ev[c.nev - 1]) == cudaSuccess) {
      for (int s = 0; s + 1 < c.nev; ++s) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c.ev[s], c.ev[s + 1]) == cudaSuccess) avg_ms[s] += ms;
      }
      *nsegments = std::max(*nsegments, c.nev - 1);
      ++*ncalls;
    }
    for (int k = 0; k < c.nev; ++k) cudaEventDestroy(c.ev[k]);
  }
  plan->timed.swap(keep);
  if (*ncalls > 0)
    for (int s = 0; s < kMaxStages; ++s) avg_ms[s] /= (float)*ncalls;
  return GBFFT_OK;
}

// ------------------------------------------------------------- plan cache

static std::mutex g_cache_mu;
static std::map<std::tuple<int, int, int, int, int, int, int, unsigned>, gbfft_plan> g_cache;

int gbfft_plan_get_cached(gbfft_plan* out, int nx, int ny, int nz, int kind, int dtype, int batch,
                          unsigned flags) {
  if (!out) return GBFFT_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return GBFFT_ERR_NO_DEVICE;
  }
  auto key = std::make_tuple(dev, nx, ny, nz, kind, dtype, batch, flags);
  std::lock_guard<std::mutex> lk(g_cache_mu);
  auto it = g_cache.find(key);
  if (it != g_cache.end()) {
    *out = it->second;
    return GBFFT_OK;
  }
  gbfft_plan p = nullptr;
  int rc = gbfft_plan_create(&p, nx, ny, nz, kind, dtype, batch, flags);
  if (rc) {
    *out = nullptr;
    return rc;
  }
  g_cache[key] = p;
  *out = p;
  return GBFFT_OK;
}

void gbfft_plan_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  for (auto& kv : g_cache) free_plan(kv.second);
  g_cache.clear();
}

}  // extern "C"

// ------------------------------------------------------- batched grids

namespace gbfft {
void register_many_group_0(std::vector<ManyKernel>&);
void register_many_group_1(std::vector<ManyKernel>&);
std::vector<ManyKernel>& many_registry() {
  static std::vector<ManyKernel> v;
  return v;
}
static std::once_flag g_many_once;
static const ManyKernel* find_many(const std::vector<int>& codes) {
  std::call_once(g_many_once, [] {
    register_many_group_0(many_registry());
    register_many_group_1(many_registry());
  });
  for (const auto& k : many_registry()) {
    bool all = true;
    for (int c : codes) {
      bool f = false;
      for (int i = 0; i < k.ncodes; ++i) f |= k.codes[i] == c;
      all &= f;
    }
    if (all) return &k;
  }
  return nullptr;
}
// Tiles per ticket a length allows: 1, 2, 4 while a team of 256 / S threads
// still covers threads_for(L) (the 16-pencil tile's natural block size).
static int many_max_teams(int L) {
  int s = 1;
  while (s < 4 && (kManyThreads / (2 * s)) >= threads_for(L)) s *= 2;
  return s;
}
}  // namespace gbfft

struct gbfft_many_s {
  int count = 0, device = 0;
  unsigned flags = 0;
  std::vector<gbfft_plan> plans;  // one per grid: twiddles, and the separate-launch path
  std::vector<long long> offs;    // element offset of each grid in the packed buffers
  long long total = 0;            // complex elements of all grids
  // host copy of the segments of each pipeline (forward, inverse), stage-major, teams = 1
  std::vector<ManySegment> base[2];
  // tuning: tiles per ticket of each axis length (index L <= 256), per pipeline
  int teams_by_len[2][257];
  // queue lag of the one launch: stage s of grid g takes slot g + s * lag
  int lag[2] = {1, 1};
  bool tuned[2] = {false, false};
  float tuned_ms[2] = {0.f, 0.f};
  // device tables, rebuilt by many_upload when the tuning changes
  ManySegment* segs[2] = {nullptr, nullptr};  // stage-major (one launch per stage)
  unsigned int* first[2] = {nullptr, nullptr};
  unsigned char* tile_seg[2] = {nullptr, nullptr};
  // the one-launch queue's order: stage s of grid g at slot g + s (see many_upload)
  ManySegment* segs_q[2] = {nullptr, nullptr};
  unsigned int* first_q[2] = {nullptr, nullptr};
  unsigned char* tile_seg_q[2] = {nullptr, nullptr};
  std::vector<unsigned int> first_host[2];
  unsigned int tiles[2] = {0, 0};  // tickets of a launch (all stages)
  unsigned int max_tickets[2] = {0, 0};  // device table capacity (teams = 1)
  int nseg = 0;
  const ManyKernel* kern[2] = {nullptr, nullptr};
  void* ws = nullptr;
  void* ws2 = nullptr;
  Control* ctl = nullptr;
  unsigned int* counters = nullptr;
  size_t counter_words = 0;
};

static void free_many(gbfft_many_s* m) {
  if (!m) return;
  for (auto p : m->plans) free_plan(p);
  for (int i = 0; i < 2; ++i) {
    cudaFree(m->segs[i]);
    cudaFree(m->first[i]);
    cudaFree(m->tile_seg[i]);
    cudaFree(m->segs_q[i]);
    cudaFree(m->first_q[i]);
    cudaFree(m->tile_seg_q[i]);
  }
  cudaFree(m->ws);
  cudaFree(m->ws2);
  cudaFree(m->ctl);
  delete m;
}

// Build and upload the device tables of pipeline `pipe` for the current
// tuning: every segment's team count, its tickets (tiles / S, rounded up), the
// stage-major ticket prefix sums of the per-stage launches and the diagonal
// queue order of the one-launch schedule: stage s of grid g at slot
// g + s * lag (lag 1: z of grid t-2, y of grid t-1, x of grid t share slot
// t). Every dependency still has a smaller ticket, and only a few grids are
// in flight at a time, whose intermediates (tens of MB) stay in L2 between
// their stages; a longer lag queues a consumer further behind its producer.
// Synchronous (plain copies): not for use during stream capture.
static int many_upload(gbfft_many_s* m, int pipe) {
  const int count = m->count;
  std::vector<ManySegment> segs = m->base[pipe];
  std::vector<unsigned int> first;
  std::vector<int> codes;
  unsigned int acc = 0;
  for (auto& sg : segs) {
    const int L = sg.d.L;
    sg.teams = (L <= 256) ? m->teams_by_len[pipe][L] : 1;
    if (sg.teams != 1 && sg.teams != 2 && sg.teams != 4) sg.teams = 1;
    first.push_back(acc);
    acc += (unsigned int)((sg.d.n_tiles + sg.teams - 1) / sg.teams);
    const int code = many_code(L, sg.d.dir, sg.teams);
    if (std::find(codes.begin(), codes.end(), code) == codes.end()) codes.push_back(code);
  }
  first.push_back(acc);
  const ManyKernel* k = find_many(codes);
  if (!k) return GBFFT_ERR_UNSUPPORTED_SIZE;
  std::vector<ManySegment> segs_q;
  std::vector<unsigned int> first_q;
  unsigned int accq = 0;
  const int lag = m->lag[pipe];
  for (int slot = 0; slot < count + 2 * lag; ++slot)
    for (int st = 2; st >= 0; --st) {
      const int g = slot - st * lag;
      if (g < 0 || g >= count) continue;
      const ManySegment& sg = segs[(size_t)st * count + g];
      first_q.push_back(accq);
      accq += (unsigned int)((sg.d.n_tiles + sg.teams - 1) / sg.teams);
      segs_q.push_back(sg);
    }
  first_q.push_back(accq);
  if (acc > m->max_tickets[pipe] || accq != acc) return GBFFT_ERR_INVALID_ARG;
  std::vector<unsigned char> ts(acc), tsq(acc);
  for (size_t sg = 0; sg + 1 < first.size(); ++sg)
    for (unsigned t = first[sg]; t < first[sg + 1]; ++t) ts[t] = (unsigned char)sg;
  for (size_t sg = 0; sg + 1 < first_q.size(); ++sg)
    for (unsigned t = first_q[sg]; t < first_q[sg + 1]; ++t) tsq[t] = (unsigned char)sg;
  const size_t sb = segs.size() * sizeof(ManySegment), fb = first.size() * sizeof(unsigned int);
  bool ok = cudaMemcpy(m->segs[pipe], segs.data(), sb, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(m->first[pipe], first.data(), fb, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(m->segs_q[pipe], segs_q.data(), sb, cudaMemcpyHostToDevice) == cudaSuccess &&
            cudaMemcpy(m->first_q[pipe], first_q.data(), fb, cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok && acc > 0)
    ok = cudaMemcpy(m->tile_seg[pipe], ts.data(), acc, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(m->tile_seg_q[pipe], tsq.data(), acc, cudaMemcpyHostToDevice) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return GBFFT_ERR_CUDA;
  }
  m->first_host[pipe] = first;
  m->tiles[pipe] = acc;
  m->kern[pipe] = k;
  return GBFFT_OK;
}

extern "C" {

int gbfft_many_create(gbfft_many* out, int count, const int* dims, int kind, int dtype, unsigned flags) {
  if (!out) return GBFFT_ERR_INVALID_ARG;
  *out = nullptr;
  if (count < 1 || 3 * count > kManyMaxSegs || !dims) return GBFFT_ERR_INVALID_ARG;
  if (kind != GBFFT_C2C || dtype != GBFFT_FP32) return GBFFT_ERR_INVALID_ARG;  // batching is built for C2C FP32
  if (flags & ~(unsigned)GBFFT_DEBUG_TIMEOUT) return GBFFT_ERR_INVALID_ARG;
  gbfft_many_s* m = new gbfft_many_s();
  m->count = count;
  m->flags = flags;
  cudaGetDevice(&m->device);
  for (int pipe = 0; pipe < 2; ++pipe)
    for (int L = 0; L <= 256; ++L) m->teams_by_len[pipe][L] = 1;
  size_t words = 0;
  for (int g = 0; g < count; ++g) {
    gbfft_plan p = nullptr;
    int rc = gbfft_plan_create(&p, dims[3 * g], dims[3 * g + 1], dims[3 * g + 2], GBFFT_C2C, GBFFT_FP32, 1,
                               GBFFT_STAGED | (flags & GBFFT_DEBUG_TIMEOUT));
    if (rc) {
      free_many(m);
      return rc;
    }
    m->plans.push_back(p);
    m->offs.push_back(m->total);
    long long n = (long long)dims[3 * g] * dims[3 * g + 1] * dims[3 * g + 2];
    m->total += (n + 1) / 2 * 2;  // keep every grid 16-byte aligned
  }
  // segments stage-major: every grid's first stage, then second, then third
  for (int pipe = 0; pipe < 2; ++pipe) {
    const int op = pipe == 0 ? GBFFT_OP_FORWARD : GBFFT_OP_INVERSE;
    std::vector<Pipeline> P(count);
    const Buf none{nullptr, -1};
    for (int g = 0; g < count; ++g) {
      // every stage of grid g must stay inside grid g's slice of the packed buffers
      const long long ng = (long long)dims[3 * g] * dims[3 * g + 1] * dims[3 * g + 2];
      char* fake = reinterpret_cast<char*>(16);  // non-null placeholder, never dereferenced
      const Buf b{fake, ng};
      Pipeline chk = build_pipeline(m->plans[g], pipe, op, b, b, b, b);
      if (validate(chk) != GBFFT_OK) {
        free_many(m);
        return GBFFT_ERR_INVALID_ARG;
      }
      P[g] = build_pipeline(m->plans[g], pipe, op, none, none, none, none);
    }
    // in -> ws, ws -> ws2, ws2 -> out: no stage of a grid overwrites a buffer an earlier stage of the grid
    // read or wrote, so the one launch needs no ordering beyond each tile's producers (with out as the
    // middle buffer, the last stage would overwrite it while middle-stage tiles still read it)
    const int roles[3][2] = {{0, 2}, {2, 3}, {3, 1}};
    std::vector<ManySegment>& segs = m->base[pipe];
    unsigned int acc = 0;
    for (int k = 0; k < 3; ++k)
      for (int g = 0; g < count; ++g) {
        ManySegment sg;
        std::memset(&sg, 0, sizeof(sg));
        sg.d = P[g].st[k];
        sg.d.in = nullptr;
        sg.d.out = nullptr;
        sg.in_buf = roles[k][0];
        sg.out_buf = roles[k][1];
        sg.in_off = m->offs[g];
        sg.out_off = m->offs[g];
        sg.teams = 1;
        sg.c_outer = (long long)words;
        words += (size_t)sg.d.batch * sg.d.n_outer;
        sg.c_outer16 = (long long)words;
        words += (size_t)sg.d.batch * gchunks(sg.d.n_outer);
        sg.c_gchunk = (long long)words;
        words += (size_t)sg.d.batch * sg.d.n_gchunks;
        sg.c_total = (long long)words;
        words += (size_t)sg.d.batch;
        sg.c_stage = (long long)words;
        words += 1;
        sg.p_outer = sg.p_outer16 = sg.p_gchunk = sg.p_total = sg.p_stage = -1;
        sg.prev_tiles = 0;
        if (k > 0) {
          const ManySegment& q = segs[(size_t)(k - 1) * count + g];
          sg.p_outer = q.c_outer;
          sg.p_outer16 = q.c_outer16;
          sg.p_gchunk = q.c_gchunk;
          sg.p_total = q.c_total;
          sg.p_stage = q.c_stage;
          sg.prev_tiles = q.d.n_tiles;
        }
        acc += (unsigned int)sg.d.n_tiles;
        segs.push_back(sg);
      }
    // each segment publishes only the counters its consumer (next stage, same grid) waits on
    for (int k = 0; k + 1 < 3; ++k)
      for (int g = 0; g < count; ++g) {
        ManySegment& sg = segs[(size_t)k * count + g];
        const int rule = segs[(size_t)(k + 1) * count + g].d.dep_rule;
        sg.sig_mask = kSigStage | (rule == kDepGroup ? kSigOuter16 : 0) | (rule == kDepGchunkOfOuter ? kSigGchunk : 0);
      }
    m->max_tickets[pipe] = acc;
  }
  m->nseg = 3 * count;
  m->counter_words = words;  // forward and inverse counters are laid out side by side
  bool ok = true;
  for (int pipe = 0; pipe < 2 && ok; ++pipe) {
    const size_t sb = m->base[pipe].size() * sizeof(ManySegment);
    const size_t fb = (m->base[pipe].size() + 1) * sizeof(unsigned int);
    const size_t tb = std::max<size_t>(m->max_tickets[pipe], 1);
    ok = cudaMalloc(&m->segs[pipe], sb) == cudaSuccess && cudaMalloc(&m->first[pipe], fb) == cudaSuccess &&
         cudaMalloc(&m->tile_seg[pipe], tb) == cudaSuccess && cudaMalloc(&m->segs_q[pipe], sb) == cudaSuccess &&
         cudaMalloc(&m->first_q[pipe], fb) == cudaSuccess && cudaMalloc(&m->tile_seg_q[pipe], tb) == cudaSuccess;
  }
  void* c = nullptr;
  ok = ok && cudaMalloc(&m->ws, (size_t)m->total * sizeof(float2)) == cudaSuccess &&
       cudaMalloc(&m->ws2, (size_t)m->total * sizeof(float2)) == cudaSuccess &&
       cudaMalloc(&c, sizeof(Control) + m->counter_words * sizeof(unsigned int)) == cudaSuccess &&
       cudaMemset(c, 0, sizeof(Control) + m->counter_words * sizeof(unsigned int)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    if (c) cudaFree(c);
    free_many(m);
    return GBFFT_ERR_ALLOC;
  }
  m->ctl = reinterpret_cast<Control*>(c);
  m->counters = reinterpret_cast<unsigned int*>(reinterpret_cast<char*>(c) + sizeof(Control));
  for (int pipe = 0; pipe < 2; ++pipe) {
    int rc = many_upload(m, pipe);
    if (rc) {
      free_many(m);
      return rc;
    }
  }
  *out = m;
  return GBFFT_OK;
}

int gbfft_many_layout(gbfft_many m, int grid, long long* offset, long long* total) {
  if (!m || grid < 0 || grid >= m->count) return GBFFT_ERR_INVALID_ARG;
  if (offset) *offset = m->offs[grid];
  if (total) *total = m->total;
  return GBFFT_OK;
}

}  // extern "C"

static int many_launch(gbfft_many m, int op, const void* in, void* out, void* stream, bool queue) {
  if (!m || (op != GBFFT_OP_FORWARD && op != GBFFT_OP_INVERSE)) return GBFFT_ERR_INVALID_ARG;
  int rc = check_ptrs(in, out);
  if (rc) return rc;
  if (cudaSetDevice(m->device) != cudaSuccess) return GBFFT_ERR_CUDA;
  const int pipe = op == GBFFT_OP_FORWARD ? 0 : 1;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  ManyArgs a;
  std::memset(&a, 0, sizeof(a));
  a.segs = queue ? m->segs_q[pipe] : m->segs[pipe];
  a.first = queue ? m->first_q[pipe] : m->first[pipe];
  a.tile_seg = queue ? m->tile_seg_q[pipe] : m->tile_seg[pipe];
  a.nseg = m->nseg;
  a.total = m->tiles[pipe];
  a.in = reinterpret_cast<const float2*>(in);
  a.out = reinterpret_cast<float2*>(out);
  a.ws = reinterpret_cast<float2*>(m->ws);
  a.ws2 = reinterpret_cast<float2*>(m->ws2);
  a.ctl = m->ctl;
  a.counters = m->counters;
  const bool dbg = (m->flags & GBFFT_DEBUG_TIMEOUT) != 0;
  a.timeout_ns = dbg ? 20000000LL : 2000000000LL;
  a.debug_never = dbg ? 1 : 0;
  const ManyKernel* k = m->kern[pipe];
  int bpsm = 1;
  cudaError_t e = launch_info(k->fn, kManyThreads, k->smem, &bpsm);
  if (e != cudaSuccess) return GBFFT_ERR_CUDA;
  a.queue = queue ? 1 : 0;
  if (queue) {
    e = cudaMemsetAsync(&m->ctl->ticket, 0, 2 * sizeof(unsigned int) + m->counter_words * sizeof(unsigned int), st);
    if (e != cudaSuccess) return GBFFT_ERR_CUDA;
    // one block per ticket; every block a block waits for has started
    void* args[] = {&a};
    e = cudaLaunchKernel(k->fn, dim3((unsigned)std::max<unsigned>(a.total, 1u)), dim3(kManyThreads), args, k->smem,
                         st);
    return cuda_err(e);
  }
  // one launch per stage over every grid's tickets of that stage
  for (int stg = 0; stg < 3; ++stg) {
    const unsigned lo = m->first_host[pipe][(size_t)stg * m->count];
    const unsigned hi = m->first_host[pipe][(size_t)(stg + 1) * m->count];
    if (hi <= lo) continue;
    a.ticket_base = lo;
    a.total = hi;
    void* args[] = {&a};
    e = cudaLaunchKernel(k->fn, dim3(hi - lo), dim3(kManyThreads), args, k->smem, st);
    if (e != cudaSuccess) return GBFFT_ERR_CUDA;
  }
  return GBFFT_OK;
}

extern "C" {

int gbfft_many_exec(gbfft_many m, int op, const void* in, void* out, void* stream) {
  return many_launch(m, op, in, out, stream, true);
}

int gbfft_many_exec_staged(gbfft_many m, int op, const void* in, void* out, void* stream) {
  return many_launch(m, op, in, out, stream, false);
}

int gbfft_many_exec_separate(gbfft_many m, int op, const void* in, void* out, void* stream) {
  if (!m || (op != GBFFT_OP_FORWARD && op != GBFFT_OP_INVERSE)) return GBFFT_ERR_INVALID_ARG;
  int rc = check_ptrs(in, out);
  if (rc) return rc;
  for (int g = 0; g < m->count; ++g) {
    rc = gbfft_exec(m->plans[g], op, reinterpret_cast<const float2*>(in) + m->offs[g],
                    reinterpret_cast<float2*>(out) + m->offs[g], stream);
    if (rc) return rc;
  }
  return GBFFT_OK;
}

// Distinct axis lengths of pipeline `pipe`, largest total tile count first.
static std::vector<int> many_lengths(const gbfft_many_s* m, int pipe) {
  std::vector<std::pair<long long, int>> w;
  for (const auto& sg : m->base[pipe]) {
    auto it = std::find_if(w.begin(), w.end(), [&](const std::pair<long long, int>& x) { return x.second == sg.d.L; });
    if (it == w.end()) w.push_back({sg.d.n_tiles, sg.d.L});
    else it->first += sg.d.n_tiles;
  }
  std::sort(w.begin(), w.end(), [](const std::pair<long long, int>& a, const std::pair<long long, int>& b) {
    return a.first > b.first;
  });
  std::vector<int> out;
  for (auto& x : w) out.push_back(x.second);
  return out;
}

int gbfft_many_autotune(gbfft_many m, void* stream) {
  if (!m) return GBFFT_ERR_INVALID_ARG;
  if (cudaSetDevice(m->device) != cudaSuccess) return GBFFT_ERR_CUDA;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  void *x = nullptr, *y = nullptr;
  const size_t bytes = (size_t)std::max<long long>(m->total, 2) * sizeof(float2);
  if (cudaMalloc(&x, bytes) != cudaSuccess || cudaMalloc(&y, bytes) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(x);
    return GBFFT_ERR_ALLOC;
  }
  int rc = cuda_err(cudaMemsetAsync(x, 0, bytes, st));
  const int reps = 5;
  for (int pipe = 0; pipe < 2 && !rc; ++pipe) {
    const int op = pipe == 0 ? GBFFT_OP_FORWARD : GBFFT_OP_INVERSE;
    auto run = [&] { return many_launch(m, op, x, y, st, true); };
    for (int L = 0; L <= 256; ++L) m->teams_by_len[pipe][L] = 1;
    m->lag[pipe] = 1;
    rc = many_upload(m, pipe);
    if (rc) break;
    float best = time_calls(run, st, reps);
    if (best < 0.f) {
      rc = GBFFT_ERR_CUDA;
      break;
    }
    // coordinate descent over the lengths, two sweeps: each length's tiles per ticket in turn
    for (int sweep = 0; sweep < 2 && !rc; ++sweep)
      for (int L : many_lengths(m, pipe)) {
        const int keep = m->teams_by_len[pipe][L];
        int best_s = keep;
        for (int S = 1; S <= many_max_teams(L); S *= 2) {
          if (S == keep) continue;
          m->teams_by_len[pipe][L] = S;
          rc = many_upload(m, pipe);
          if (rc) break;
          const float t = time_calls(run, st, reps);
          if (t >= 0.f && t < best) {
            best = t;
            best_s = S;
          }
        }
        if (rc) break;
        m->teams_by_len[pipe][L] = best_s;
      }
    // queue lag between a grid's stages
    for (int lag : {2, 4, 8}) {
      if (rc) break;
      const int keep = m->lag[pipe];
      m->lag[pipe] = lag;
      rc = many_upload(m, pipe);
      if (rc) break;
      const float t = time_calls(run, st, reps);
      if (t >= 0.f && t < best) best = t;
      else m->lag[pipe] = keep;
    }
    if (!rc) rc = many_upload(m, pipe);
    m->tuned[pipe] = rc == GBFFT_OK;
    m->tuned_ms[pipe] = best;
  }
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(x);
  cudaFree(y);
  if (!rc && e != cudaSuccess) rc = GBFFT_ERR_CUDA;
  return rc;
}

int gbfft_many_get_tuning(gbfft_many m, int pipeline, int* lengths, int* teams, int cap, int* n, float* ms) {
  if (!m || pipeline < 0 || pipeline > 1 || !n || cap < 0) return GBFFT_ERR_INVALID_ARG;
  const std::vector<int> ls = many_lengths(m, pipeline);
  *n = (int)ls.size();
  for (int i = 0; i < (int)ls.size() && i < cap; ++i) {
    if (lengths) lengths[i] = ls[i];
    if (teams) teams[i] = m->teams_by_len[pipeline][ls[i]];
  }
  if (ms) *ms = m->tuned[pipeline] ? m->tuned_ms[pipeline] : 0.f;
  return GBFFT_OK;
}

int gbfft_many_get_lag(gbfft_many m, int pipeline, int* lag) {
  if (!m || pipeline < 0 || pipeline > 1 || !lag) return GBFFT_ERR_INVALID_ARG;
  *lag = m->lag[pipeline];
  return GBFFT_OK;
}

int gbfft_many_set_lag(gbfft_many m, int pipeline, int lag) {
  if (!m || pipeline < 0 || pipeline > 1 || lag < 1 || lag > 8) return GBFFT_ERR_INVALID_ARG;
  if (cudaSetDevice(m->device) != cudaSuccess) return GBFFT_ERR_CUDA;
  m->lag[pipeline] = lag;
  return many_upload(m, pipeline);
}

int gbfft_many_set_tuning(gbfft_many m, int pipeline, const int* lengths, const int* teams, int n) {
  if (!m || pipeline < 0 || pipeline > 1 || n < 0 || (n > 0 && (!lengths || !teams))) return GBFFT_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    if (lengths[i] < 2 || lengths[i] > 256) return GBFFT_ERR_INVALID_ARG;
    if (teams[i] != 1 && teams[i] != 2 && teams[i] != 4) return GBFFT_ERR_INVALID_ARG;
    if (teams[i] > many_max_teams(lengths[i])) return GBFFT_ERR_INVALID_ARG;
  }
  if (cudaSetDevice(m->device) != cudaSuccess) return GBFFT_ERR_CUDA;
  for (int i = 0; i < n; ++i) m->teams_by_len[pipeline][lengths[i]] = teams[i];
  return many_upload(m, pipeline);
}

int gbfft_many_get_device_error(gbfft_many m, int* code) {
  if (!m || !code) return GBFFT_ERR_INVALID_ARG;
  if (cudaSetDevice(m->device) != cudaSuccess) return GBFFT_ERR_CUDA;
  if (cudaDeviceSynchronize() != cudaSuccess) return GBFFT_ERR_CUDA;
  int e = 0;
  if (cudaMemcpy(&e, &m->ctl->error, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return GBFFT_ERR_CUDA;
  *code = e == kDevErrTimeout ? GBFFT_ERR_TIMEOUT : (e ? GBFFT_ERR_CUDA : GBFFT_OK);
  if (cudaMemset(&m->ctl->error, 0, sizeof(int)) != cudaSuccess) return GBFFT_ERR_CUDA;
  return GBFFT_OK;
}

void gbfft_many_destroy(gbfft_many m) { free_many(m); }

}  // extern "C"
