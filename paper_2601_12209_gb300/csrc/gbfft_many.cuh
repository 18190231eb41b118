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
//
// Tile shape (Section III-C's granularity trade-off, chosen per axis length
// by the batched plan's autotuner): a ticket of a segment carries S = 1, 2 or
// 4 tiles of 16 pencils, run side by side by S teams of 256 / S threads. At
// the short lengths one 16-pencil tile keeps only 32-128 threads busy and a
// block's fixed cost (ticket, descriptor, twiddles, dependency wait, release)
// is paid per tile; S tiles per ticket fill the block and share that cost.
#pragma once
#include "gbfft_kernels.cuh"

namespace gbfft {

// One stage of one grid. d.in / d.out are unused; the kernel rebuilds them as
// base[in_buf] + in_off and base[out_buf] + out_off.
struct ManySegment {
  StageDesc d;
  int in_buf, out_buf;  // 0 in, 1 out, 2 and 3 the two workspaces
  // counters the consumer segment reads (kSig* bits); the others are not written
  int sig_mask;
  int teams;  // S: tiles per ticket (1, 2 or 4), one team of kManyThreads / S threads each
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
  float2* ws2;
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

// Kernel code of a batched stage: kcode(L, kPlain, dir) with the team count S in bits 24-26.
constexpr int many_code(int L, int dir, int S) { return kcode(L, kPlain, dir) | (S << 24); }
__host__ __device__ constexpr int many_code_len(int c) { return (c >> 8) & 0xFFFF; }
__host__ __device__ constexpr int many_code_teams(int c) { return c >> 24; }

// Rows of shared tile the kernel needs: S tiles of L + 1 rows (16 pencils each).
template <int CODE, int... REST>
__host__ __device__ constexpr int many_max_rows() {
  constexpr int r = many_code_teams(CODE) * (many_code_len(CODE) + 1);
  if constexpr (sizeof...(REST) == 0) return r;
  else return r > many_max_rows<REST...>() ? r : many_max_rows<REST...>();
}

template <int CODE, int... REST>
__host__ __device__ constexpr int many_max_tw() {
  constexpr int t = tw_table_len(many_code_len(CODE));
  if constexpr (sizeof...(REST) == 0) return t;
  else return t > many_max_tw<REST...>() ? t : many_max_tw<REST...>();
}

template <int... CODES>
constexpr size_t many_smem_bytes() {
  return sizeof(float2) * ((size_t)many_max_rows<CODES...>() * kTileP + (size_t)((many_max_tw<CODES...>() + 7) / 8 * 8));
}

// Run ticket t0 of a segment with code `code`: team j of the block takes tile t0 * S + j (idle past the end).
template <int CODE, int... REST>
__device__ __forceinline__ void many_dispatch(int code, const StageDesc& d, long long t0, float2* sm, const float2* tw) {
  if (code == CODE) {
    constexpr int L = many_code_len(CODE), S = many_code_teams(CODE), DIR = (CODE & 1) ? 1 : -1;
    constexpr int TT = kManyThreads / S;
    const int team = (int)threadIdx.x / TT;
    const long long tile = t0 * S + team;
    const bool idle = tile >= d.n_tiles;
    process_tile<L, DIR, kPlain, TT>(d, idle ? t0 * S : tile, sm + team * (L + 1) * kTileP, tw, tw, idle);
  } else if constexpr (sizeof...(REST) > 0) {
    many_dispatch<REST...>(code, d, t0, sm, tw);
  }
}

__device__ __forceinline__ bool many_wait_tile(const ManyArgs& a, const ManySegment& m, long long tile) {
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

// Waits for the producer tiles of every tile of ticket t0. (The stages of a
// grid write three distinct buffers, ws, ws2 and out, so no stage overwrites
// what an earlier stage read or wrote: the producer tiles are the only order
// a tile needs.)
__device__ __forceinline__ bool many_wait(const ManyArgs& a, const ManySegment& m, long long t0) {
  for (int j = 0; j < m.teams; ++j) {
    const long long tile = t0 * m.teams + j;
    if (tile >= m.d.n_tiles) break;
    if (!many_wait_tile(a, m, tile)) return false;
  }
  return true;
}

__device__ __forceinline__ void many_signal_tile(const ManyArgs& a, const ManySegment& m, long long tile) {
  const StageDesc& d = m.d;
  // 32-bit decode (tile counts stay below 2^32): 64-bit division is a subroutine call
  const unsigned t32 = (unsigned)tile;
  const unsigned gc = t32 % (unsigned)d.n_gchunks;
  const unsigned rest = t32 / (unsigned)d.n_gchunks;
  const int o = (int)(rest % (unsigned)d.n_outer);
  const int b = (int)(rest / (unsigned)d.n_outer);
  const int n16 = (d.n_outer + kTileP - 1) / kTileP;
  unsigned int* C = a.counters;
  if (m.sig_mask & kSigOuter16) atomicAdd(C + m.c_outer16 + (long long)b * n16 + o / kTileP, 1u);
  if (m.sig_mask & kSigGchunk) atomicAdd(C + m.c_gchunk + (long long)b * d.n_gchunks + gc, 1u);
}

// Publishes every tile of ticket t0 (the stage counter once, by the ticket's tile count).
__device__ __forceinline__ void many_signal(const ManyArgs& a, const ManySegment& m, long long t0) {
  if (!m.sig_mask) return;  // last stage of its grid: nobody waits on it
  // release fence: the block's stores (observed through the barrier) before the counter updates
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  unsigned int n = 0;
  for (int j = 0; j < m.teams; ++j) {
    const long long tile = t0 * m.teams + j;
    if (tile >= m.d.n_tiles) break;
    many_signal_tile(a, m, tile);
    ++n;
  }
  if (m.sig_mask & kSigStage) atomicAdd(a.counters + m.c_stage, n);
}

// One ticket per block: the block takes the next ticket, finds its segment,
// waits (bounded) for the producer tiles it reads, runs the tile and
// publishes it. Blocks are launched in ticket order, so every tile a block
// waits for belongs to a block that is already running (no deadlock). One
// straight-line tile per block also keeps the eleven lengths' butterflies in
// registers (inside a tile loop the compiler spills them).
template <int... CODES>
__global__ void __launch_bounds__(kManyThreads, 3) many_kernel(ManyArgs a) {
  extern __shared__ float4 smem4[];
  float2* sm = reinterpret_cast<float2*>(smem4);
  float2* tw = sm + many_max_rows<CODES...>() * kTileP;  // 16-byte aligned: rows * 16 float2
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
      const float2* bases_in[4] = {a.in, a.out, a.ws, a.ws2};
      float2* bases_out[4] = {const_cast<float2*>(a.in), a.out, a.ws, a.ws2};
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
  many_dispatch<CODES...>(stage_code(s_seg.d) | (s_seg.teams << 24), s_seg.d, s_tile, sm, tw);
  __syncthreads();
  if (a.queue && threadIdx.x == 0) many_signal(a, s_seg, s_tile);
}

struct ManyKernel {
  int ncodes;
  int codes[32];
  const void* fn;
  size_t smem;
};

template <int... CODES>
ManyKernel make_many_entry() {
  ManyKernel k{};
  const int codes[] = {CODES...};
  static_assert(sizeof...(CODES) <= 32, "ManyKernel holds up to 32 codes");
  k.ncodes = (int)sizeof...(CODES);
  for (int i = 0; i < k.ncodes; ++i) k.codes[i] = codes[i];
  k.fn = reinterpret_cast<const void*>(&many_kernel<CODES...>);
  k.smem = many_smem_bytes<CODES...>();
  return k;
}

std::vector<ManyKernel>& many_registry();

}  // namespace gbfft
