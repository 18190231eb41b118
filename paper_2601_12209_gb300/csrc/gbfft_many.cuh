// Batched persistent kernel: many C2C grids of different sizes in ONE launch.
//
// The paper's runtime spawns every chunk task of every stage into one task
// graph and lets ready tasks run wherever a worker is free (Sections III-C,
// IV-C/D); the benefit it reports is largest when chunk costs are uneven
// (Table II). Here the tasks of all grids share one ticket counter. The
// queue orders segments diagonally (stage s of grid g at slot g + s), so each
// dependency has a smaller ticket, a grid's y tiles start as soon as that
// grid's x planes are done, whatever the other grids are doing, and the few
// grids in flight keep their intermediates in L2. The per-stage launches over
// all grids (no waits) use the stage-major order of the same segments.
//
// Segments (one stage of one grid) live in device memory with buffer-relative
// addresses, so a launch needs only the in / out / workspace base pointers and
// can be captured in a CUDA graph and replayed.
#pragma once
#include "gbfft_kernels.cuh"

namespace gbfft {

// One stage of one grid. d.in / d.out are unused; the kernel rebuilds them as
// base[in_buf] + in_off and base[out_buf] + out_off.
struct ManySegment {
  StageDesc d;
  int in_buf, out_buf;  // 0 in, 1 out, 2 workspace
  // counters the consumer segment reads (kSig* bits); the others are not written
  int sig_mask, sig_pad;
  long long in_off, out_off;
  // counters of this segment (offsets into the launch's counter buffer)
  long long c_outer, c_outer16, c_gchunk, c_total, c_stage;
  // counters of the producer segment (same grid, previous stage); -1 if none
  long long p_outer, p_outer16, p_gchunk, p_total, p_stage;
  long long prev_tiles;  // tiles of the producer segment
};

struct ManyArgs {
  const ManySegment* segs;
  const unsigned int* first;  // nseg + 1 prefix sums of tiles
  const unsigned char* tile_seg;  // segment of every ticket
  int nseg;
  unsigned int total;
  const float2* in;
  float2* out;
  float2* ws;
  Control* ctl;
  unsigned int* counters;
  long long timeout_ns;
  int debug_never;
  // queue = 1: blocks take tickets from ctl->ticket and wait on dependencies
  // (all stages in one launch); queue = 0: block b runs ticket ticket_base + b
  // with no waits (one launch per stage, kernel boundaries order the stages)
  int queue;
  unsigned int ticket_base;
};

constexpr int kSigOuter16 = 1, kSigGchunk = 2, kSigStage = 4;
constexpr int kManyThreads = 256;
constexpr int kManyMaxSegs = 256;  // 3 stages x up to 85 grids per launch

template <int CODE, int... REST>
__host__ __device__ constexpr int many_max_len() {
  if constexpr (sizeof...(REST) == 0) return CODE >> 8;
  else return (CODE >> 8) > many_max_len<REST...>() ? (CODE >> 8) : many_max_len<REST...>();
}

template <int... CODES>
constexpr size_t many_smem_bytes() {
  constexpr int LM = many_max_len<CODES...>();
  return sizeof(float2) * ((size_t)(LM + 1) * kTileP + (size_t)((max_tw_len<CODES...>() + 7) / 8 * 8));
}

__device__ __forceinline__ bool many_wait(const ManyArgs& a, const ManySegment& m, long long tile) {
  const StageDesc& d = m.d;
  if (m.p_stage < 0 || d.dep_rule == kDepNone) return true;
  const unsigned int extra = a.debug_never ? 1u : 0u;
  unsigned int* C = a.counters;
  if (ld_acquire(C + m.p_stage) >= (unsigned int)m.prev_tiles + extra) return true;
  // 32-bit decode (tile counts stay below 2^32): 64-bit division is a subroutine call
  const unsigned t32 = (unsigned)tile;
  const unsigned gc = t32 % (unsigned)d.n_gchunks;
  const unsigned rest = t32 / (unsigned)d.n_gchunks;
  const int o = (int)(rest % (unsigned)d.n_outer);
  const int b = (int)(rest / (unsigned)d.n_outer);
  const unsigned long long t0 = global_ns();
  switch (d.dep_rule) {
    case kDepGroup: {
      const int n16 = (d.prev_n_outer + kTileP - 1) / kTileP;
      const int outers = min(kTileP, d.prev_n_outer - (int)gc * kTileP);
      return wait_counter(C + m.p_outer16 + (long long)b * n16 + gc,
                          (unsigned int)(outers * d.prev_n_gchunks) + extra, a.ctl, a.timeout_ns, t0);
    }
    case kDepGchunkOfOuter:
      return wait_counter(C + m.p_gchunk + (long long)b * d.prev_n_gchunks + o / kTileP,
                          (unsigned int)d.prev_n_outer + extra, a.ctl, a.timeout_ns, t0);
    default:
      return wait_counter(C + m.p_stage, (unsigned int)m.prev_tiles + extra, a.ctl, a.timeout_ns, t0);
  }
}

__device__ __forceinline__ void many_signal(const ManyArgs& a, const ManySegment& m, long long tile) {
  const StageDesc& d = m.d;
  // 32-bit decode (tile counts stay below 2^32): 64-bit division is a subroutine call
  const unsigned t32 = (unsigned)tile;
  const unsigned gc = t32 % (unsigned)d.n_gchunks;
  const unsigned rest = t32 / (unsigned)d.n_gchunks;
  const int o = (int)(rest % (unsigned)d.n_outer);
  const int b = (int)(rest / (unsigned)d.n_outer);
  const int n16 = (d.n_outer + kTileP - 1) / kTileP;
  unsigned int* C = a.counters;
  if (!m.sig_mask) return;  // last stage of its grid: nobody waits on it
  __threadfence();
  if (m.sig_mask & kSigOuter16) atomicAdd(C + m.c_outer16 + (long long)b * n16 + o / kTileP, 1u);
  if (m.sig_mask & kSigGchunk) atomicAdd(C + m.c_gchunk + (long long)b * d.n_gchunks + gc, 1u);
  if (m.sig_mask & kSigStage) atomicAdd(C + m.c_stage, 1u);
}

// One ticket per block: the block takes the next ticket, finds its segment,
// waits (bounded) for the producer tiles it reads, runs the tile and
// publishes it. Blocks are launched in ticket order, so every tile a block
// waits for belongs to a block that is already running (no deadlock). One
// straight-line tile per block also keeps the eleven lengths' butterflies in
// registers (inside a tile loop the compiler spills them).
template <int... CODES>
__global__ void __launch_bounds__(kManyThreads, 3) many_kernel(ManyArgs a) {
  constexpr int LM = many_max_len<CODES...>();
  extern __shared__ float4 smem4[];
  float2* sm = reinterpret_cast<float2*>(smem4);
  float2* tw = sm + (LM + 1) * kTileP;  // 16-byte aligned: (LM + 1) * 16 float2
  __shared__ __align__(16) ManySegment s_seg;
  __shared__ long long s_tile;
  __shared__ unsigned int s_t;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    const unsigned int t = a.queue ? atomicAdd(&a.ctl->ticket, 1u) : a.ticket_base + blockIdx.x;
    s_t = t;
    s_ok = (t < a.total && !(a.queue && *reinterpret_cast<volatile int*>(&a.ctl->abort))) ? 1 : 0;
  }
  __syncthreads();
  if (!s_ok) return;
  const unsigned int t = s_t;
  const int seg = a.tile_seg[t];
  if (threadIdx.x < 32) {  // warp 0 copies the segment descriptor, 8 bytes per lane
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(a.segs + seg);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&s_seg);
    for (int i = threadIdx.x; i < (int)(sizeof(ManySegment) / 8); i += 32) dst[i] = src[i];
    __syncwarp();
    if (threadIdx.x == 0) {
      const float2* bases_in[3] = {a.in, a.out, a.ws};
      float2* bases_out[3] = {const_cast<float2*>(a.in), a.out, a.ws};
      s_seg.d.in = bases_in[s_seg.in_buf] + s_seg.in_off;
      s_seg.d.out = bases_out[s_seg.out_buf] + s_seg.out_off;
      s_tile = (long long)(t - a.first[seg]);
      if (a.queue && !many_wait(a, s_seg, s_tile)) {
        atomicCAS(&a.ctl->error, 0, kDevErrTimeout);
        atomicExch(&a.ctl->abort, 1);
        s_ok = 0;
      }
    }
  }
  __syncthreads();
  if (!s_ok) return;
  for (int i = threadIdx.x; i < s_seg.d.tw_len; i += kManyThreads) tw[i] = s_seg.d.tw[i];
  __syncthreads();
  dispatch_tile<kManyThreads, CODES...>(stage_code(s_seg.d), s_seg.d, s_tile, sm, tw, tw);
  __syncthreads();
  if (a.queue && threadIdx.x == 0) many_signal(a, s_seg, s_tile);
}

struct ManyKernel {
  int ncodes;
  int codes[16];
  const void* fn;
  size_t smem;
};

template <int... CODES>
ManyKernel make_many_entry() {
  ManyKernel k{};
  const int codes[] = {CODES...};
  k.ncodes = (int)sizeof...(CODES);
  for (int i = 0; i < k.ncodes; ++i) k.codes[i] = codes[i];
  k.fn = reinterpret_cast<const void*>(&many_kernel<CODES...>);
  k.smem = many_smem_bytes<CODES...>();
  return k;
}

std::vector<ManyKernel>& many_registry();

}  // namespace gbfft
