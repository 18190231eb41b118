// Kernel templates: one launch per stage (stage_kernel) and one persistent
// launch for a whole transform (persistent_kernel), plus the registry entries
// the host dispatches through.
#pragma once
#include <vector>

#include "gbfft_device.cuh"
#include "gbfft_warp_tile.cuh"

namespace gbfft {

// ------------------------------------------------------------- registry

struct StageKernel {
  int L, dir, kind;
  int prec;  // StagePrec of the radix-16 passes
  const void* fn;
  int threads;
  size_t smem;
  bool loops;  // grid-stride tile loop (else one tile per block)
};

struct PersistentKernel {
  int ncodes;
  int codes[8];  // (L << 8) | (kind << 1) | (dir > 0)
  const void* fn;
  int threads;
  bool warp_body;  // its length-512 complex stages can run the warp-per-pencil tile body (StageDesc::body)
  size_t smem;               // tile bytes
  size_t tw_smem_per_stage;  // twiddle bytes per stage (total = smem + nstages * this)
};

// A TMA stage kernel (gbfft_tma.cuh): input tiles arrive by tensor copies.
// Tensor-copy boxes (shared by the kernels and the host's tensor maps)
constexpr int kRowBoxN = 16;  // transform indices per row-side box
constexpr int kColBoxN = 8;   // transform indices per column-side box (one 1 KB swizzle atom)

struct TmaKernel {
  int L, dir, kind, src;  // src: 1 row-side copies, 2 column-side copies
  const void* fn;
  int threads;
  size_t smem;
};

constexpr int kcode(int L, int kind, int dir) { return (L << 8) | (kind << 1) | (dir > 0 ? 1 : 0); }

std::vector<StageKernel>& stage_registry();
std::vector<PersistentKernel>& persistent_registry();
std::vector<TmaKernel>& tma_registry();

// --------------------------------------------------------- stage kernel

template <int L, int KIND>
constexpr size_t stage_smem_bytes() {
  return sizeof(float2) * ((size_t)(L + 1) * kTileP + tw_table_len(L) + (L + 1));
}

// Power-of-two lengths: each block loops over tiles with a grid stride, so the
// twiddle tables are staged into shared memory once per block. Mixed-radix
// lengths (factors 3, 5): one tile per block -- inside a tile loop the
// compiler's register allocation of their butterflies spills, straight-line
// it does not; the hardware block scheduler then hands out the tiles.
__host__ __device__ constexpr bool stage_loops(int L) { return (L & (L - 1)) == 0; }

// Programmatic dependent launch. Stage kernels are launched so that they may
// start while the previous kernel in the stream drains: every block lets the
// next grid launch (its blocks take SM slots as this grid's blocks retire, and
// only once every block of this grid has started), runs its prologue (the
// twiddle tables of the plan), then waits until the previous grid has
// completed and its writes are visible before it reads its input.
__device__ __forceinline__ void pdl_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait_prev() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// The tensor-core passes hold a column group's accumulators across the
// pass's barrier as well as the DFT-16 operand fragments: one block fewer.
__host__ __device__ constexpr int stage_min_blocks(int L, int prec) {
  return prec == kPrecFP32 ? min_blocks_for(L) : (min_blocks_for(L) > 1 ? min_blocks_for(L) - 1 : 1);
}

// Block size of a stage kernel: threads_for(L), except that the tensor-core
// passes at length 1024 keep 512 threads (their accumulators and operand
// fragments do not fit the 64 registers of a 1024-thread block).
__host__ __device__ constexpr int stage_threads(int L, int prec) {
  return (prec != kPrecFP32 && L >= 1024) ? 512 : threads_for(L);
}

template <int L, int DIR, int KIND, int PREC = kPrecFP32>
__global__ void __launch_bounds__(stage_threads(L, PREC), stage_min_blocks(L, PREC)) stage_kernel(StageDesc d) {
  constexpr int THREADS = stage_threads(L, PREC);
  extern __shared__ float4 smem4[];
  float2* sm = reinterpret_cast<float2*>(smem4);
  float2* tw = sm + (L + 1) * kTileP;
  constexpr int TWL = tw_table_len(L);
  float2* tw2 = tw + TWL;
  pdl_launch_next();
  load_twiddles<L, THREADS>(tw, tw2, d, KIND == kR2CPost || KIND == kC2RPre || KIND >= kPoissonZB);
  if constexpr (prec_is_tc5(PREC)) tc5_setup<L, DIR, PREC, THREADS>(d.err);  // tensor memory, B operands
  __syncthreads();
  pdl_wait_prev();
  if constexpr (stage_loops(L) && KIND == kC2RPre && PREC == kPrecFP32) {
    if (d.in_mode == kCol && static_cast<const void*>(d.in) != static_cast<const void*>(d.out)) {
      // C2R from the column side: the first loads of the block's next tile are
      // issued before this tile's row store, so their latency overlaps the store
      C2REarlyLoads<L, THREADS> r;
      bool have = false;  // r holds the early loads of `tile`
      for (long long tile = blockIdx.x; tile < d.n_tiles; tile += gridDim.x) {
        int o, g0;
        const TileIO io = make_io(d, tile, o, g0);
        if (pair_vec_ok(io.gin, io.in_n, io.valid)) {
          if (!have) c2r_issue_early<L, THREADS>(io, r);
          c2r_merge_rest<L, THREADS>(sm, tw2, d.interior, io, r);
        } else {
          col_load_c2r_pre<L, THREADS>(sm, tw2, d.interior, io);
        }
        fft_passes<L, +1, THREADS, false, false, false>(sm, tw, io);
        have = false;
        const long long next = tile + gridDim.x;
        if (next < d.n_tiles) {
          const TileIO nio = make_io(d, next, o, g0);
          if (pair_vec_ok(nio.gin, nio.in_n, nio.valid)) {
            c2r_issue_early<L, THREADS>(nio, r);
            have = true;
          }
        }
        row_store<THREADS, L>(sm, io);
        __syncthreads();
      }
      return;
    }
  }
  if constexpr (stage_loops(L)) {
    for (long long tile = blockIdx.x; tile < d.n_tiles; tile += gridDim.x) {
      process_tile<L, DIR, KIND, THREADS, PREC>(d, tile, sm, tw, tw2);
      __syncthreads();
    }
  } else {
    if ((long long)blockIdx.x < d.n_tiles)
      process_tile<L, DIR, KIND, THREADS, PREC>(d, (long long)blockIdx.x, sm, tw, tw2);
  }
  if constexpr (prec_is_tc5(PREC)) tc5_teardown<L>();
}

template <int L, int DIR, int KIND, int PREC = kPrecFP32>
StageKernel make_stage_entry() {
  return StageKernel{L, DIR, KIND, PREC, reinterpret_cast<const void*>(&stage_kernel<L, DIR, KIND, PREC>),
                     stage_threads(L, PREC), stage_smem_bytes<L, KIND>(), stage_loops(L)};
}

// ----------------------------------------------------- persistent kernel
//
// The paper's dynamic scheduler hands ready DTasks to idle workers
// (Sections III-C, IV-C/D). Here every block is a worker: it takes the next
// ticket from one atomic counter (tickets are the stages' tiles, stage after
// stage, so every dependency has a smaller ticket), waits (bounded) until the
// tiles it reads are complete, runs the tile, and publishes its completion on
// counters -- the per-chunk dependency tracking of DataDepsTaskQueue
// (Section IV-D) with counters instead of task graphs. Each worker fetches
// its next ticket while it works on the current one, and stops checking a
// stage's dependencies once the whole producer stage is known complete.

struct PersistentArgs {
  StageDesc st[kMaxStages];
  int nstages;
  unsigned int total;                    // tickets = sum of the stages' tiles
  Control* ctl;
  unsigned int* cnt_outer[kMaxStages];   // per (batch, outer index)
  unsigned int* cnt_outer16[kMaxStages]; // per (batch, outer index / 16)
  unsigned int* cnt_gchunk[kMaxStages];  // per (batch, group chunk)
  unsigned int* cnt_total[kMaxStages];   // per batch entry
  unsigned int* cnt_stage[kMaxStages];   // one per stage
  long long timeout_ns;                  // bound on every dependency wait
  int debug_never;                       // wait for one more completion than exists (timeout test)
  // counters a stage's tiles publish: the one the next stage's rule waits on
  // and the stage total (kPSig* bits); 0 for the last stage (nobody waits)
  int sig[kMaxStages];
  // consecutive tiles of one stage per ticket (1, 2 or 4): the ticket, the
  // dependency look-ahead and the publishing fence are paid once per ticket
  int tiles_per_ticket;
  // war[s] >= 0: stage s writes a buffer that stage war[s] (< s) read or wrote,
  // so its tiles first wait for that whole stage (write-after-read / -write:
  // the dependency rules order only the producer tiles a tile reads); -1: none
  int war[kMaxStages];
};

constexpr int kMaxTicketTiles = 4;

constexpr int kPSigOuter = 1, kPSigOuter16 = 2, kPSigGchunk = 4, kPSigTotal = 8, kPSigStage = 16;

// The counters stage s + 1 reads under its dependency rule (plus the stage total,
// which every wait checks first).
__host__ __device__ constexpr int persistent_sig_for_rule(int rule) {
  return kPSigStage | (rule == kDepGroup ? kPSigOuter16 : 0) | (rule == kDepOuter ? kPSigOuter : 0) |
         (rule == kDepGchunkOfOuter || rule == kDepSameGchunk ? kPSigGchunk : 0) | (rule == kDepAll ? kPSigTotal : 0);
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned int ld_relaxed(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait until *p >= target. Returns false on timeout or abort.
__device__ __forceinline__ bool wait_counter(const unsigned int* p, unsigned int target, Control* ctl,
                                             long long timeout_ns, unsigned long long t0) {
  unsigned int spins = 0;
  while (ld_acquire(p) < target) {
    if ((++spins & 15) == 0) {
      if (*reinterpret_cast<volatile int*>(&ctl->abort)) return false;
      if ((long long)(global_ns() - t0) > timeout_ns) return false;
    }
    __nanosleep(100);
  }
  return true;
}

// The counter tile `tile` of stage s waits on under its stage's rule, and the
// count it waits for (*target); nullptr when it waits for nothing (first
// stage, no rule, or the producer stage already known complete).
__device__ __forceinline__ const unsigned int* dep_counter(const PersistentArgs& a, const StageDesc* st,
                                                          const int* complete, int s, long long tile,
                                                          unsigned int* target) {
  if (s == 0) return nullptr;
  const StageDesc& d = st[s];
  if (d.dep_rule == kDepNone || complete[s - 1]) return nullptr;
  const unsigned int extra = a.debug_never ? 1u : 0u;
  // 32-bit decode (tile counts stay below 2^32): 64-bit division is a subroutine call
  const unsigned t32 = (unsigned)tile;
  const unsigned gc = t32 % (unsigned)d.n_gchunks;
  const unsigned rest = t32 / (unsigned)d.n_gchunks;
  const int o = (int)(rest % (unsigned)d.n_outer);
  const int b = (int)(rest / (unsigned)d.n_outer);
  switch (d.dep_rule) {
    case kDepGroup: {
      // the consumer's group chunk gc is the producer's outer chunk gc
      const int n16 = (d.prev_n_outer + kTileP - 1) / kTileP;
      const int outers = min(kTileP, d.prev_n_outer - (int)gc * kTileP);
      *target = (unsigned int)(outers * d.prev_n_gchunks) + extra;
      return a.cnt_outer16[s - 1] + (long long)b * n16 + gc;
    }
    case kDepOuter:
      *target = (unsigned int)d.prev_n_gchunks + extra;
      return a.cnt_outer[s - 1] + (long long)b * d.prev_n_outer + o;
    case kDepGchunkOfOuter:
      *target = (unsigned int)d.prev_n_outer + extra;
      return a.cnt_gchunk[s - 1] + (long long)b * d.prev_n_gchunks + o / kTileP;
    case kDepSameGchunk:
      *target = (unsigned int)d.prev_n_outer + extra;
      return a.cnt_gchunk[s - 1] + (long long)b * d.prev_n_gchunks + gc;
    case kDepAll:
      *target = (unsigned int)(d.prev_n_outer * d.prev_n_gchunks) + extra;
      return a.cnt_total[s - 1] + b;
  }
  return nullptr;
}

// Wait for the producer tiles (previous stage) that tile `tile` of stage s reads.
// One counter per rule; `complete` caches "the whole previous stage is done".
__device__ __forceinline__ bool wait_deps(const PersistentArgs& a, const StageDesc* st, int* complete, int s,
                                          long long tile) {
  if (s == 0) return true;
  const unsigned int extra = a.debug_never ? 1u : 0u;
  const int w = a.war[s];
  if (w >= 0 && !complete[w]) {
    // the whole earlier stage that touched this stage's output buffer
    if (!wait_counter(a.cnt_stage[w], (unsigned int)st[w].n_tiles + extra, a.ctl, a.timeout_ns, global_ns()))
      return false;
    complete[w] = 1;
  }
  const StageDesc& d = st[s];
  if (d.dep_rule == kDepNone || complete[s - 1]) return true;
  if (ld_acquire(a.cnt_stage[s - 1]) >= (unsigned int)st[s - 1].n_tiles + extra) {
    complete[s - 1] = 1;
    return true;
  }
  unsigned int target = 0;
  const unsigned int* p = dep_counter(a, st, complete, s, tile, &target);
  return p ? wait_counter(p, target, a.ctl, a.timeout_ns, global_ns()) : true;
}

// Publish ntiles finished tiles from tile0 on. Called by one thread after a block barrier: the
// fence orders the whole block's stores (observed through the barrier) before
// the counter updates that consumers acquire.
__device__ __forceinline__ void signal_done(const PersistentArgs& a, const StageDesc* st, int s, long long tile0,
                                            int ntiles) {
  const StageDesc& d = st[s];
  const int sig = a.sig[s];
  if (!sig) return;  // last stage of the launch: nobody waits on it
  // release fence: the block's stores (observed through the barrier) before the
  // counter updates, which consumers read with ld.acquire
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  const int n16 = (d.n_outer + kTileP - 1) / kTileP;
  for (int j = 0; j < ntiles; ++j) {
    // 32-bit decode (tile counts stay below 2^32): 64-bit division is a subroutine call
    const unsigned t32 = (unsigned)(tile0 + j);
    const unsigned gc = t32 % (unsigned)d.n_gchunks;
    const unsigned rest = t32 / (unsigned)d.n_gchunks;
    const int o = (int)(rest % (unsigned)d.n_outer);
    const int b = (int)(rest / (unsigned)d.n_outer);
    if (sig & kPSigOuter) atomicAdd(a.cnt_outer[s] + (long long)b * d.n_outer + o, 1u);
    if (sig & kPSigOuter16) atomicAdd(a.cnt_outer16[s] + (long long)b * n16 + o / kTileP, 1u);
    if (sig & kPSigGchunk) atomicAdd(a.cnt_gchunk[s] + (long long)b * d.n_gchunks + gc, 1u);
    if (sig & kPSigTotal) atomicAdd(a.cnt_total[s] + b, 1u);
  }
  if (sig & kPSigStage) atomicAdd(a.cnt_stage[s], (unsigned int)ntiles);
}

// Runtime dispatch of one tile over the compile-time list of (L, kind, dir)
// codes this kernel was built for.
// A length-512 complex stage of a 512-thread persistent block may run the
// warp-per-pencil body instead (d.body = 1): its twiddle block then holds
// W_L^(t k1) [k1][t] (L entries) and W_32^(c k2') (32 entries) instead of the
// packed Stockham table.
__host__ __device__ constexpr bool persistent_warp_body(int threads, int L, int kind) {
  return threads == kWarpThreads && L == 512 && kind == kPlain;
}

template <int THREADS, int CODE, int... REST>
__device__ __forceinline__ void dispatch_tile(int code, const StageDesc& d, long long tile, float2* sm,
                                              const float2* tw, const float2* tw2) {
  if (code == CODE) {
    constexpr int L = CODE >> 8, KIND = (CODE >> 1) & 127, DIR = (CODE & 1) ? 1 : -1;
    if constexpr (persistent_warp_body(THREADS, L, KIND)) {
      if (d.body) {
        warp_tile<L, DIR, KIND>(d, tile, sm, tw, tw + L, tw2);
        return;
      }
    }
    process_tile<L, DIR, KIND, THREADS>(d, tile, sm, tw, tw2);
  } else if constexpr (sizeof...(REST) > 0) {
    dispatch_tile<THREADS, REST...>(code, d, tile, sm, tw, tw2);
  }
}

template <int CODE, int... REST>
__host__ __device__ constexpr int max_len() {
  if constexpr (sizeof...(REST) == 0) return CODE >> 8;
  else return (CODE >> 8) > max_len<REST...>() ? (CODE >> 8) : max_len<REST...>();
}

template <int CODE, int... REST>
__host__ __device__ constexpr int min_threads() {
  if constexpr (sizeof...(REST) == 0) return threads_for(CODE >> 8);
  else return threads_for(CODE >> 8) < min_threads<REST...>() ? threads_for(CODE >> 8) : min_threads<REST...>();
}

// Block size of a persistent family: the smallest natural block size of its
// lengths, so the register budget of the longest length is not cut down to
// what twice as many threads would allow (the longer stages then run more
// butterflies per thread).
template <int... CODES>
__host__ __device__ constexpr int family_threads() {
  return min_threads<CODES...>();
}

// Shared memory of a persistent launch: the tile, then one twiddle block
// (W_L, and W_2L for real transforms) per stage of the launch.
// Tile rows of the warp-per-pencil body (16 padded pencil regions) where a
// family's block can run it, else 0.
template <int THREADS, int CODE, int... REST>
__host__ __device__ constexpr int persistent_warp_rows() {
  constexpr int L = CODE >> 8;
  constexpr int r = persistent_warp_body(THREADS, L, (CODE >> 1) & 127) ? kTileP * WarpGeom<512>::kRegion : 0;
  if constexpr (sizeof...(REST) == 0) return r;
  else return r > persistent_warp_rows<THREADS, REST...>() ? r : persistent_warp_rows<THREADS, REST...>();
}

template <int... CODES>
__host__ __device__ constexpr size_t persistent_tile_bytes() {
  constexpr int stockham = (max_len<CODES...>() + 1) * kTileP;
  constexpr int warp = persistent_warp_rows<family_threads<CODES...>(), CODES...>();
  return sizeof(float2) * (size_t)(stockham > warp ? stockham : warp);
}
template <int CODE, int... REST>
__host__ __device__ constexpr int max_tw_len() {
  if constexpr (sizeof...(REST) == 0) return tw_table_len(CODE >> 8);
  else return tw_table_len(CODE >> 8) > max_tw_len<REST...>() ? tw_table_len(CODE >> 8) : max_tw_len<REST...>();
}

// per stage: the packed twiddles, then W_2L (real transforms); a multiple of
// 8 entries so every stage's table starts 64-byte aligned (the butterflies
// read twiddle pairs as 16-byte loads)
template <int... CODES>
__host__ __device__ constexpr int persistent_tw_block() {
  return (max_tw_len<CODES...>() + max_len<CODES...>() + 1 + 7) / 8 * 8;
}
template <int... CODES>
constexpr size_t persistent_tw_bytes_per_stage() {
  return sizeof(float2) * (size_t)persistent_tw_block<CODES...>();
}

__device__ __forceinline__ int stage_code(const StageDesc& d) {
  return (d.L << 8) | (d.kind << 1) | (d.dir > 0 ? 1 : 0);
}

template <int... CODES>
__global__ void __launch_bounds__(family_threads<CODES...>(), min_blocks_for(max_len<CODES...>()))
persistent_kernel(PersistentArgs a) {
  constexpr int THREADS = family_threads<CODES...>();
  extern __shared__ float4 smem4[];
  float2* sm = reinterpret_cast<float2*>(smem4);
  // twiddle blocks after the tile, which is the larger of the Stockham tile and the warp-per-pencil regions
  constexpr int kTileF2 = (int)(persistent_tile_bytes<CODES...>() / sizeof(float2));
  static_assert(kTileF2 % 8 == 0, "every stage's twiddle block starts 64-byte aligned");
  float2* tws = sm + kTileF2;
  __shared__ StageDesc s_st[kMaxStages];
  __shared__ unsigned int s_first[kMaxStages + 1];
  __shared__ int s_complete[kMaxStages];
  __shared__ unsigned int s_ticket;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    unsigned int acc = 0;
#pragma unroll
    for (int k = 0; k < kMaxStages; ++k) {
      s_st[k] = a.st[k];
      s_first[k] = acc;
      s_complete[k] = 0;
      if (k < a.nstages) acc += (unsigned int)((a.st[k].n_tiles + a.tiles_per_ticket - 1) / a.tiles_per_ticket);
    }
    s_first[kMaxStages] = acc;
    s_ticket = atomicAdd(&a.ctl->ticket, 1u);
  }
  __syncthreads();
  constexpr int TWB = persistent_tw_block<CODES...>();
  constexpr int TW2 = max_tw_len<CODES...>();
  static_assert(persistent_warp_rows<THREADS, CODES...>() == 0 || TW2 >= 512 + 32,
                "the warp-per-pencil tables of a stage fit below its W_2L table");
  for (int s = 0; s < a.nstages; ++s) {
    float2* tw = tws + s * TWB;
    const StageDesc& d = s_st[s];
    if (d.body) {  // warp-per-pencil tables (length 512: R1 = 16)
      for (int i = threadIdx.x; i < d.L; i += THREADS) tw[i] = d.twn[(i & 31) * (i >> 5)];
      if (threadIdx.x < 32) tw[d.L + threadIdx.x] = d.twn[(16 * (threadIdx.x / 16) * (threadIdx.x % 16)) % d.L];
    } else {
      for (int i = threadIdx.x; i < d.tw_len; i += THREADS) tw[i] = d.tw[i];
    }
    if (d.kind == kR2CPost || d.kind == kC2RPre)
      for (int i = threadIdx.x; i <= d.L; i += THREADS) tw[TW2 + i] = d.tw2[i];
  }
  __syncthreads();
  // Worker loop with a look-ahead of one ticket. A ticket is T consecutive
  // tiles of one stage (T = a.tiles_per_ticket). Thread 0 holds the ticket
  // after the current one (t1) and fetches the one after that (t2) while the
  // block works; at the start of a ticket it also reads the counters t1's
  // tiles wait on (relaxed loads, then an acquire fence). When they are already
  // complete the block starts t1 after this ticket without a block barrier,
  // while thread 0 publishes the finished tiles; otherwise thread 0 publishes
  // them and then waits (bounded) for t1's producers before the block goes on. Every tile is published before its block waits for
  // anything, so every wait is for tiles of blocks that are running. Slot
  // (iteration & 1) of s_tk / s_go is written by thread 0 one iteration ahead
  // of its readers.
  const int T = a.tiles_per_ticket;
  __shared__ unsigned int s_tk[2];
  __shared__ int s_go[2];
  unsigned int t1 = 0, t2 = 0;
  if (threadIdx.x == 0) {
    s_tk[0] = s_ticket;
    s_go[0] = 0;
    t1 = atomicAdd(&a.ctl->ticket, 1u);
  }
  __syncthreads();
  for (int it = 0;; ++it) {
    const int slot = it & 1;
    const unsigned int t = s_tk[slot];
    if (t >= a.total) break;
    int s = 0;
    while (s + 1 < a.nstages && t >= s_first[s + 1]) ++s;
    const long long tile0 = (long long)(t - s_first[s]) * T;
    const long long ntiles = s_st[s].n_tiles;
    if (!s_go[slot]) {
      if (threadIdx.x == 0) {
        int ok = *reinterpret_cast<volatile int*>(&a.ctl->abort) ? 0 : 1;
        for (int j = 0; j < T && ok && tile0 + j < ntiles; ++j) {
          if (!wait_deps(a, s_st, s_complete, s, tile0 + j)) {
            atomicCAS(&a.ctl->error, 0, kDevErrTimeout);
            atomicExch(&a.ctl->abort, 1);
            ok = 0;
          }
        }
        s_ok = ok;
      }
      __syncthreads();
      if (!s_ok) break;
    }
    // look ahead (thread 0): are the next ticket's producers complete? Its answer goes to the next
    // slot now; the loads hold back only thread 0, once per ticket.
    if (threadIdx.x == 0) {
      int go = 1;
      if (t1 < a.total) {
        int s1 = 0;
        while (s1 + 1 < a.nstages && t1 >= s_first[s1 + 1]) ++s1;
        const long long u0 = (long long)(t1 - s_first[s1]) * T;
        const unsigned int* lp[kMaxTicketTiles] = {nullptr, nullptr, nullptr, nullptr};
        unsigned int lv[kMaxTicketTiles] = {0, 0, 0, 0}, lt[kMaxTicketTiles] = {0, 0, 0, 0};
        bool any = false;
#pragma unroll
        for (int j = 0; j < kMaxTicketTiles; ++j)
          if (j < T && u0 + j < s_st[s1].n_tiles) {
            lp[j] = dep_counter(a, s_st, s_complete, s1, u0 + j, &lt[j]);
            if (lp[j]) {
              lv[j] = ld_relaxed(lp[j]);
              any = true;
            }
          }
        // the whole earlier stage whose buffer the next ticket's stage overwrites
        const int w = s1 > 0 ? a.war[s1] : -1;
        const bool wchk = w >= 0 && !s_complete[w];
        const unsigned int wv = wchk ? ld_relaxed(a.cnt_stage[w]) : 0u;
        any = any || wchk;
        if (any) asm volatile("fence.acq_rel.gpu;" ::: "memory");  // acquire: the loads above, then the tiles
#pragma unroll
        for (int j = 0; j < kMaxTicketTiles; ++j)
          if (lp[j] && lv[j] < lt[j]) go = 0;
        if (wchk && wv < (unsigned int)s_st[w].n_tiles + (a.debug_never ? 1u : 0u)) go = 0;
      }
      t2 = atomicAdd(&a.ctl->ticket, 1u);  // needed one ticket later
      s_tk[slot ^ 1] = t1;
      s_go[slot ^ 1] = (t1 >= a.total || go) ? 1 : 0;
    }
    const StageDesc& d = s_st[s];
    const float2* tw = tws + s * TWB;
    for (int j = 0; j < T && tile0 + j < ntiles; ++j) {
      if (j > 0) __syncthreads();  // the previous tile of the ticket is out of shared memory
      dispatch_tile<THREADS, CODES...>(stage_code(d), d, tile0 + j, sm, tw, tw + TW2);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      signal_done(a, s_st, s, tile0, (int)min((long long)T, ntiles - tile0));
      t1 = t2;
    }
  }
}

template <int... CODES>
PersistentKernel make_persistent_entry() {
  PersistentKernel k{};
  const int codes[] = {CODES...};
  k.ncodes = (int)sizeof...(CODES);
  for (int i = 0; i < k.ncodes; ++i) k.codes[i] = codes[i];
  k.fn = reinterpret_cast<const void*>(&persistent_kernel<CODES...>);
  k.threads = family_threads<CODES...>();
  k.warp_body = persistent_warp_rows<family_threads<CODES...>(), CODES...>() > 0;
  k.smem = persistent_tile_bytes<CODES...>();
  k.tw_smem_per_stage = persistent_tw_bytes_per_stage<CODES...>();
  return k;
}

}  // namespace gbfft
