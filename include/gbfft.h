/*
 * gbfft -- staged 3D FFT for one GB300 (sm_103a): C ABI.
 *
 * The operation (arxiv 2601.12209, Section III-A): for A of size
 * Nx x Ny x Nz,
 *   A^(kx,ky,kz) = sum_{i,j,l} A(i,j,l) exp(-2 pi i (kx i/Nx + ky j/Ny + kz l/Nz)),
 * evaluated as the paper's pencil sequence: Ny*Nz length-Nx transforms, a
 * redistribution, Nx*Nz length-Ny transforms, a redistribution, Nx*Ny
 * length-Nz transforms (Section III-A; Algorithm 1). The slab variant
 * (Section III-A) transforms x and y plane by plane before one redistribution
 * and the z transforms. The inverse mirrors the sequence (Section IV-A).
 *
 * Layout. Arrays are row-major [batch][nz][ny][nx] (x fastest), the same
 * element order as the paper's column-major A(i,j,l) with i = x fastest.
 * Complex data is interleaved float32 (re, im) -- complex64. For
 * GBFFT_R2C plans the real array is [batch][nz][ny][nx] float32 and the
 * spectrum is [batch][nz][ny][nx/2+1] complex64 (the x axis is halved).
 *
 * Conventions (readings of the paper, which states no normalisation):
 *   forward  : sign -, unscaled
 *   inverse  : sign +, scaled by 1/(nx ny nz), so inverse(forward(x)) = x
 *   adjoint  : conjugate transpose of forward (sign +, no scaling); for R2C,
 *              the transpose of the real-to-complex map
 *   inverse_adjoint : transpose of inverse (= forward / N for C2C)
 * The C2R direction uses only the Hermitian part of the kx = 0 and kx = nx/2
 * planes (the imaginary parts there are projected out).
 *
 * Ownership and memory. `in` and `out` are device pointers owned by the
 * caller, contiguous, 16-byte aligned, and must not overlap (out-of-place;
 * `in` is never written). The plan owns its twiddle tables, schedules and,
 * unless gbfft_set_workspace is called, its workspace.
 *
 * Asynchrony. exec calls enqueue work on `stream` (a cudaStream_t, NULL =
 * legacy default stream) and return without synchronising. Device-side
 * errors (a dependency wait that timed out) are reported by
 * gbfft_get_device_error. A plan may be used from one stream at a time.
 *
 * Errors. Every function returns 0 on success or a negative GBFFT_ERR_*
 * code; nothing throws across this interface.
 */
#ifndef GBFFT_H
#define GBFFT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbfft_plan_s* gbfft_plan;

/* transform kinds (Section V-B: C2C and R2C; C2R is the inverse of R2C) */
#define GBFFT_C2C 0
#define GBFFT_R2C 1

/* arithmetic: storage is always float32 / complex64 */
#define GBFFT_FP32 0
/* Storage stays complex64 in every mode; the radix-16 passes run as dense
 * 16x16 DFT products on the tensor cores with each FP32 operand split into a
 * hi/lo pair of FP16 (or BF16) values, three products per term, FP32
 * accumulation, and a power-of-two scale per butterfly. Not in the paper: an
 * extension of its per-axis 1D FFT step (Section III-A). The complex stages
 * take them (every stage of a C2C plan; the y and z stages of an R2C plan,
 * whose real x stage and fused Poisson z stage keep FP32); axes whose length
 * has no radix-16 pass (or is 16 itself, a half-warp kernel) keep the FP32
 * butterflies. */
#define GBFFT_FP16_SPLIT 1
#define GBFFT_BF16_SPLIT 2
/* The same split products on the 5th-generation tensor cores: tcgen05.mma
 * issued by one thread per block, operands in shared memory, FP32
 * accumulators in tensor memory, 128 butterflies per product (M = 128,
 * N = 32: the real and imaginary outputs; K = 32: the real and imaginary
 * inputs). Built for lengths whose radix-16 butterflies fill 128-row tiles
 * (128, 256, 384, 640, 768, 1024); other lengths with a radix-16 pass take
 * the warp-level (mma.sync) products of the same operand type. */
#define GBFFT_FP16_SPLIT_TC5 3
#define GBFFT_BF16_SPLIT_TC5 4

/* plan flags */
#define GBFFT_PENCIL 0u          /* three stages, two redistributions (Algorithm 1) */
#define GBFFT_SLAB 1u            /* x and y per z-plane, then z (Section III-A); the x,y pair runs
                                    as one fused plane launch where built (512^2, 256^2 planes)
                                    unless GBFFT_STAGED */
#define GBFFT_TRANSPOSED_OUT 2u  /* pencil only: forward leaves C[b][kx][ky][kz] ("collect from C",
                                    Algorithm 1); inverse then reads that layout */
#define GBFFT_STAGED 4u          /* one launch per stage instead of one persistent launch */
#define GBFFT_NO_TMA 8u          /* staged launches load tiles with thread loads instead of tensor copies */
#define GBFFT_DEBUG_TIMEOUT (1u << 16) /* tests only: every dependency wait of the persistent launch
                                          waits for one completion too many and times out after
                                          ~20 ms; gbfft_get_device_error then returns
                                          GBFFT_ERR_TIMEOUT */

/* operations for gbfft_exec */
#define GBFFT_OP_FORWARD 0
#define GBFFT_OP_INVERSE 1
#define GBFFT_OP_ADJOINT 2
#define GBFFT_OP_INVERSE_ADJOINT 3

/* error codes */
#define GBFFT_OK 0
#define GBFFT_ERR_INVALID_ARG (-1)
#define GBFFT_ERR_UNSUPPORTED_SIZE (-2) /* a length with no kernel (see gbfft_supported_length) */
#define GBFFT_ERR_ALIGNMENT (-3)        /* a pointer not 16-byte aligned */
#define GBFFT_ERR_INPLACE (-4)          /* in == out */
#define GBFFT_ERR_ALLOC (-5)            /* device allocation failed or workspace too small */
#define GBFFT_ERR_CUDA (-6)             /* a CUDA runtime call failed */
#define GBFFT_ERR_TIMEOUT (-7)          /* a device dependency wait ran out of time */
#define GBFFT_ERR_NO_DEVICE (-8)        /* no CUDA device */
#define GBFFT_ERR_STATIC_LIMIT (-9)     /* grid larger than GBFFT_NOALLOC_MAX_POINTS */
#define GBFFT_ERR_SETUP_IN_CAPTURE (-10) /* gbfft_exec_c2c_noalloc: a device's first call came while its
                                            stream was capturing (set-up needs a synchronous copy) */

/*
 * Create a plan for `batch` grids of nx x ny x nz (Section V-B: a reusable
 * plan keyed by data type, size, transform type and dimensions).
 *   kind  : GBFFT_C2C or GBFFT_R2C (R2C needs even nx)
 *   dtype : GBFFT_FP32, or GBFFT_FP16_SPLIT / GBFFT_BF16_SPLIT (and their
 *           _TC5 forms): the complex stages run stage launches without tensor
 *           copies, whatever the flags
 *   flags : GBFFT_PENCIL or GBFFT_SLAB, optionally | GBFFT_TRANSPOSED_OUT
 *           (pencil only) | GBFFT_STAGED | GBFFT_NO_TMA | GBFFT_DEBUG_TIMEOUT
 * Every axis length (nx/2 for the R2C x axis) must satisfy
 * gbfft_supported_length. Uses the current CUDA device; allocates twiddle
 * tables and schedules (and the workspace lazily, on first exec).
 * On success *out receives the plan; on failure *out is NULL.
 */
int gbfft_plan_create(gbfft_plan* out, int nx, int ny, int nz, int kind, int dtype, int batch,
                      unsigned flags);

/*
 * Plan cache (Section V-B, get_or_create_plan): returns a plan shared by all
 * callers with the same (device, nx, ny, nz, kind, dtype, batch, flags). Do
 * not destroy it; gbfft_plan_cache_clear destroys every cached plan.
 */
int gbfft_plan_get_cached(gbfft_plan* out, int nx, int ny, int nz, int kind, int dtype, int batch,
                          unsigned flags);
void gbfft_plan_cache_clear(void);

/*
 * Run one operation (GBFFT_OP_*) from `in` to `out` on `stream`.
 *   C2C: in/out complex64 [batch][nz][ny][nx] (TRANSPOSED_OUT: the forward
 *        output and the inverse input are [batch][nx][ny][nz]).
 *   R2C: FORWARD and INVERSE_ADJOINT map real -> half spectrum;
 *        INVERSE and ADJOINT map half spectrum -> real.
 */
int gbfft_exec(gbfft_plan plan, int op, const void* in, void* out, void* stream);
int gbfft_exec_forward(gbfft_plan plan, const void* in, void* out, void* stream);
int gbfft_exec_inverse(gbfft_plan plan, const void* in, void* out, void* stream);
int gbfft_exec_adjoint(gbfft_plan plan, const void* in, void* out, void* stream);
int gbfft_exec_inverse_adjoint(gbfft_plan plan, const void* in, void* out, void* stream);

/*
 * Periodic Poisson solve (Section VI-B, (Periodic, Periodic, Periodic)
 * topology): out = C2R(m * R2C(in)) / N with m(k) = -1/|k|^2, m(0) = 0, on a
 * 2 pi-periodic box (integer wavenumbers; index j > n/2 means j - n).
 * R2C plans only; in and out are real [batch][nz][ny][nx]. The multiplier
 * and the inverse z transform are fused into the forward z stage. The
 * operator is symmetric, so this call is also its own adjoint.
 */
int gbfft_exec_poisson(gbfft_plan plan, const void* in, void* out, void* stream);

/*
 * Poisson solve on the (Periodic, Periodic, Bounded) topology (Section VI-B):
 * x and y periodic as in gbfft_exec_poisson; z bounded by walls with a zero
 * normal derivative (Neumann), the nz values at cell centres of a box of
 * height pi. Along z the solve expands in cosines: DCT-II (real-to-real,
 * Section V-B) forward and DCT-III back, each computed as one length-nz
 * complex FFT, fused into the z stage with the multiplier
 * m(k) = -1/(kx^2 + ky^2 + kz^2) (kz = cosine index 0..nz-1), m(0) = 0, and
 * the normalisation 1/(2 nx ny nz). R2C plans only; in and out are real
 * [batch][nz][ny][nx]. The operator is symmetric: this call is its own adjoint.
 */
int gbfft_exec_poisson_bounded(gbfft_plan plan, const void* in, void* out, void* stream);

/* per-axis transform kinds (Section V-B: R2R transforms, DCT and DST) */
#define GBFFT_R2R_NONE (-1) /* the axis keeps its Fourier transform */
#define GBFFT_R2R_DCT 0     /* forward DCT-II (FFTW REDFT10), inverse DCT-III (REDFT01) */
#define GBFFT_R2R_DST 1     /* forward DST-II (RODFT10), inverse DST-III (RODFT01) */

/*
 * Mixed transform: along each axis (x, y, z) the DFT (GBFFT_R2R_NONE) or a
 * real-to-real transform, each computed as one length-n complex FFT inside
 * that axis's stage:
 *   DCT-II: Y_k = 2 sum_n x_n cos(pi k (2n + 1) / 2n_ax)
 *   DST-II: Y_k = 2 sum_n x_n sin(pi (k + 1) (2n + 1) / 2n_ax)
 * Forward (inverse = 0) maps the plan's forward input to its spectrum shape,
 * unscaled; inverse = 1 applies DCT-III / DST-III and inverse DFTs in reverse
 * axis order, scaled by 1 / prod(2 n_ax for R2R axes, n_ax for DFT axes), so
 * inverse(forward(x)) = x. Complex data transform their real and imaginary
 * parts alike. R2C plans keep the DFT (R2C / C2R) along x: r2r_x must be
 * GBFFT_R2R_NONE there. Pencil or slab plans; the spectrum's layout is
 * gbfft_exec_forward's (natural, or [b][kx][ky][kz] with GBFFT_TRANSPOSED_OUT).
 */
int gbfft_exec_r2r(gbfft_plan plan, int r2r_x, int r2r_y, int r2r_z, int inverse, const void* in, void* out,
                   void* stream);

/*
 * gbfft_exec_r2r(plan, GBFFT_R2R_NONE, GBFFT_R2R_NONE, r2r, ...): Fourier x and y,
 * DCT (r2r = GBFFT_R2R_DCT) or DST (GBFFT_R2R_DST) along z -- the spectral
 * basis of the (Periodic, Periodic, Bounded) topology.
 */
int gbfft_exec_r2r_z(gbfft_plan plan, int r2r, int inverse, const void* in, void* out, void* stream);

/*
 * End-to-end call on HOST buffers: copies `host_in` to the device, runs
 * `op`, copies the result to `host_out`, and waits for completion. Uses
 * plan-owned device buffers (allocated on first use). Pinned host memory
 * gives asynchronous copies. op may also be 4 for gbfft_exec_poisson, 5 for
 * gbfft_exec_poisson_bounded.
 */
int gbfft_exec_host(gbfft_plan plan, int op, const void* host_in, void* host_out);
/*
 * Split gbfft_exec_host into `chunks` slabs (1 = one copy in, the transform,
 * one copy out; 2..16) where the host array is a set of contiguous slabs: the
 * x stage that reads the rows of the input runs on slabs of z planes, each
 * after its slab's host-to-device copy, and the x stage that writes the rows
 * of the output runs on slabs whose device-to-host copies start as soon as
 * each is written; the spectrum side (read or written by the z stage, whose
 * slabs would be strided) moves in one copy. Applies to pencil plans with
 * natural output, batch 1, ops 0-3 (others take the one-copy path); the stages
 * run as stage launches with the plan's tuned per-stage kernels.
 */
int gbfft_plan_set_host_chunks(gbfft_plan plan, int chunks);

/*
 * Autotuner (Section V-B: plans pick the best execution strategy for a size
 * and transform type; Section III-C: the granularity/overhead trade-off).
 * For each pipeline of the plan -- 0 forward (FORWARD, INVERSE_ADJOINT),
 * 1 inverse (INVERSE, ADJOINT), 2 Poisson (R2C plans) -- it times on
 * `stream`, with CUDA events, every stage with each kernel family that
 * applies (thread loads, tensor copies, warp-per-pencil, the C2R kernel with
 * cp.async prefetch), the whole pipeline as one persistent launch (where a
 * kernel family exists; with 1, 2 or 4 consecutive tiles per ticket, and also
 * with the warp-per-pencil tile body on its length-512 complex stages) and, for slab plans, each in-plane stage pair as
 * one fused plane launch (a thread-block cluster per xy-plane runs both
 * stages while the plane is in L2, or, for real transforms of 512-point rows
 * with ny = 256 or 512, an 8-CTA cluster per plane keeps the plane's
 * intermediate in distributed shared memory); it keeps the fastest. Later exec calls
 * use the choice. Blocking (synchronises `stream`); allocates the plan's
 * workspace and two scratch buffers on first use; respects GBFFT_STAGED and
 * GBFFT_NO_TMA. Do not call it during stream capture.
 */
int gbfft_plan_autotune(gbfft_plan plan, void* stream);
/*
 * The tuned choice of a pipeline (0, 1, 2 as above): *tuned 0/1,
 * *persistent 0/1, *tma_mask bit s (0-7) = stage s uses the tensor-copy
 * kernel, bit 8 + s = stages s and s+1 run as one fused plane launch, bits
 * 16-19 = CTAs per plane cluster of those launches (2, 4, 8; 0 = by plane
 * size), bit 20 + s (s < 5) = stage s runs the warp-per-pencil kernel (lengths 1024, 512
 * and 256 complex, and the length-256 real x stages; FP32) -- with
 * *persistent = 1: stage s of the persistent launch runs the warp-per-pencil
 * tile body (length-512 complex stages of 512-thread families) --, bits
 * 25-26 = log2 of the persistent launch's tiles per ticket (1, 2, 4), bit
 * 27 = the fused plane launches keep the intermediate in distributed shared
 * memory (where that kernel is built; others go through L2), bit 28 + s
 * (s < 4) = stage s runs the C2R kernel with cp.async prefetch; *ms =
 * measured time of the choice, stage_ms[0..4] = per-stage times of the staged
 * candidates. Any output pointer may be NULL.
 */
int gbfft_plan_get_tuning(gbfft_plan plan, int pipeline, int* tuned, int* persistent, unsigned* tma_mask, float* ms,
                          float* stage_ms);
/*
 * Fix a pipeline's launch choice by hand (as gbfft_plan_autotune would):
 * persistent 1 = one persistent launch (when a kernel family exists; bit
 * 20 + s of tma_mask runs stage s on the warp-per-pencil tile body where it
 * can, bits 25-26 give log2 of its tiles per ticket, 3 is invalid), else
 * staged launches with bit s of tma_mask selecting the tensor-copy
 * kernel for stage s (where it applies), bit 8 + s fusing stages s and s+1
 * into one plane launch (where they are a slab plan's in-plane pair), bits
 * 16-19 the CTAs per plane cluster (2, 4 or 8; 0 = by plane size), bit 20 + s
 * the warp-per-pencil kernel for stage s (where it is built), bit 27 the
 * plane launches with the intermediate in distributed shared memory (real
 * transforms of 512-point rows, ny = 256 or 512; 8 CTAs per plane) and bit
 * 28 + s the C2R prefetch kernel for stage s (where it applies).
 */
int gbfft_plan_set_tuning(gbfft_plan plan, int pipeline, int persistent, unsigned tma_mask);
/*
 * Per-launch timing inside exec calls: while enabled, each exec records a
 * CUDA event on its stream before its first launch and after every launch.
 * gbfft_plan_stage_times synchronises on the recorded events of `pipeline`,
 * returns the average duration of each launch segment over the calls
 * (avg_ms[0..4]; one segment for a persistent launch, one per stage for
 * staged launches), the segment count and the call count, and releases them.
 */
int gbfft_plan_time_stages(gbfft_plan plan, int enable);
int gbfft_plan_stage_times(gbfft_plan plan, int pipeline, float* avg_ms, int* nsegments, int* ncalls);

/* Bytes of device workspace the plan needs (pencil: one or two spectrum-sized buffers). */
int gbfft_workspace_size(gbfft_plan plan, size_t* bytes);
/* Give the plan caller-owned workspace (>= gbfft_workspace_size bytes, 256-byte aligned). */
int gbfft_set_workspace(gbfft_plan plan, void* dev_ptr, size_t bytes);

/*
 * Read and clear the device error word of the plan's persistent launches.
 * Synchronises the device first. *code receives 0 or GBFFT_ERR_TIMEOUT.
 */
int gbfft_get_device_error(gbfft_plan plan, int* code);

/*
 * Tests only: run ONE step of the pencil pipeline with its own launch.
 *   1 stage x forward      A[b][z][y][x]  -> B[b][z][x][y]
 *   2 first redistribution alone (no arithmetic), same maps as step 1
 *   3 stage y forward      B -> C[b][x][y][z]
 *   4 second redistribution alone, same maps as step 3
 *   5 stage z forward      C -> natural [b][z][y][x]
 *   6 un-permute alone, same maps as step 5
 *  11/12 stage z inverse / its map alone:  natural -> C
 *  13/14 stage y inverse / its map alone:  C -> B
 *  15/16 stage x inverse / its map alone:  B -> A
 * Inverse steps apply no 1/N. Steps 2 and 16 need a C2C plan; for R2C plans
 * the x axis of B and C has nx/2+1 bins. The redistribution-alone steps are
 * pure moves and reproduce bit patterns exactly.
 */
int gbfft_debug_run(gbfft_plan plan, int step, const void* in, void* out, void* stream);

/*
 * Allocation-free C2C transform (the paper has no counterpart; this entry
 * point exists for callers that cannot allocate device memory when they run
 * the transform -- code whose device memory belongs to a pool or framework
 * allocator that forbids side allocations, or latency-critical loops in
 * which a cudaMalloc would synchronise the device). It needs no plan and calls no
 * cudaMalloc, cudaFree or other allocating routine: the intermediate stage
 * array lives in a file-scope static __device__ buffer of
 * GBFFT_NOALLOC_MAX_POINTS complex64 values (32 MiB) that every GPU which
 * loads this library holds until the process exits, and the twiddle tables
 * of every supported length sit in a second static array.
 *   nx, ny, nz : one grid, nx*ny*nz <= GBFFT_NOALLOC_MAX_POINTS (else
 *                GBFFT_ERR_STATIC_LIMIT, nothing launched); every length must
 *                satisfy gbfft_supported_length and be <= 1024
 *   op         : GBFFT_OP_FORWARD / INVERSE / ADJOINT / INVERSE_ADJOINT
 *   in, out    : caller-owned device buffers, complex64 [nz][ny][nx],
 *                16-byte aligned, distinct; in is not written
 *   stream     : cudaStream_t; the call enqueues three stage launches (the
 *                pencil x, y, z stages) and returns without waiting
 * The first call on a device sets that device up (resolves the static
 * arrays' device addresses, uploads the twiddle tables with a synchronous
 * copy); make that first call before any stream capture: if `stream` is
 * capturing at that point the call returns GBFFT_ERR_SETUP_IN_CAPTURE and
 * enqueues nothing. Later calls take no lock. Every stage's read and write
 * extents are checked on the host before anything is launched
 * (GBFFT_ERR_INVALID_ARG). Every call shares
 * the one scratch buffer: calls that overlap on the GPU (different streams,
 * or concurrent host threads) race on it. Nothing in it needs to start at
 * zero -- each stage writes every element before the next reads it.
 */
#define GBFFT_NOALLOC_MAX_POINTS 4194304
int gbfft_exec_c2c_noalloc(int nx, int ny, int nz, int op, const void* in, void* out, void* stream);

/*
 * Batched grids (the paper's task graph over many chunks of uneven cost,
 * Sections III-C and IV-D, Table II): `count` grids of different sizes
 * (dims[3g..3g+2] = nx, ny, nz of grid g; each length 2^a 3^b 5^c in
 * 32..256) transformed by ONE persistent launch whose blocks take the tiles of
 * every grid from one ticket counter (bounded per-grid dependency waits). The
 * grids are packed back to back in `in` and `out` (grid g starts at element
 * offset gbfft_many_layout(g); every grid starts 16-byte aligned). The launch
 * needs only in/out and plan-owned memory (two workspaces of the packed size,
 * so that no stage overwrites what an earlier stage of its grid reads), so it
 * can be captured in a CUDA graph and replayed. count <= 85.
 *   kind, dtype : as in gbfft_plan_create; batching is built for GBFFT_C2C with
 *                 GBFFT_FP32 only (any other combination: GBFFT_ERR_INVALID_ARG)
 *   flags       : 0 or GBFFT_DEBUG_TIMEOUT
 */
typedef struct gbfft_many_s* gbfft_many;
int gbfft_many_create(gbfft_many* out, int count, const int* dims, int kind, int dtype, unsigned flags);
/* Element offset of grid `grid` and the total complex elements of the packed buffers. */
int gbfft_many_layout(gbfft_many m, int grid, long long* offset, long long* total);
/* One persistent launch for all grids; op GBFFT_OP_FORWARD or GBFFT_OP_INVERSE (1/N per grid). */
int gbfft_many_exec(gbfft_many m, int op, const void* in, void* out, void* stream);
/* The same transforms as three launches, one per stage over every grid's tiles (no
   dependency waits; kernel boundaries order the stages); capturable as well. */
int gbfft_many_exec_staged(gbfft_many m, int op, const void* in, void* out, void* stream);
/* The same transforms as one plan per grid, launched one after another (for comparison). */
int gbfft_many_exec_separate(gbfft_many m, int op, const void* in, void* out, void* stream);
/*
 * Tile-shape autotuner of the batched plan (Section III-C: the granularity of
 * a task against its scheduling overhead; Section V-B: plans tuned per size).
 * A ticket of the one launch carries S = 1, 2 or 4 tiles of 16 pencils, run
 * side by side by teams of 256 / S threads: 16 S pencils per block and 16 / S
 * threads per pencil, which fills the block at the short lengths. For each
 * pipeline (0 forward, 1 inverse) and each distinct axis length the tuner
 * times the one-launch schedule on `stream` (CUDA events) for every S the
 * length allows and keeps the fastest (coordinate descent, two sweeps);
 * the per-stage launches use the same choice. Blocking; allocates two scratch
 * buffers of the packed size while it runs; not during stream capture.
 */
int gbfft_many_autotune(gbfft_many m, void* stream);
/* The tiles per ticket of pipeline 0/1: lengths[i], teams[i] for i < min(*n, cap); *n receives the
   number of distinct lengths; *ms (may be NULL) the tuned one-launch time (0 if not tuned). */
int gbfft_many_get_tuning(gbfft_many m, int pipeline, int* lengths, int* teams, int cap, int* n, float* ms);
/* Set tiles per ticket by hand (teams 1, 2 or 4, at most what the length allows; synchronous upload). */
int gbfft_many_set_tuning(gbfft_many m, int pipeline, const int* lengths, const int* teams, int n);
/* Queue lag of the one launch (chosen by gbfft_many_autotune from 1, 2, 4, 8): stage s of grid g is queued at
   slot g + s * lag, so a larger lag queues a grid's next stage further behind its producer. Every dependency
   keeps a smaller ticket for any lag. set: 1..8 (synchronous upload; not during stream capture). */
int gbfft_many_get_lag(gbfft_many m, int pipeline, int* lag);
int gbfft_many_set_lag(gbfft_many m, int pipeline, int lag);
/* Read and clear the device error word of the batched launches (synchronises). */
int gbfft_many_get_device_error(gbfft_many m, int* code);
void gbfft_many_destroy(gbfft_many m);

/* Human-readable name of an error code (static storage). */
const char* gbfft_strerror(int code);

/* Release the plan and everything it owns. NULL is ignored. */
void gbfft_plan_destroy(gbfft_plan plan);

/* ---- host-only queries (no GPU needed) ---- */

/* 1 if a pencil of length n has a compiled kernel, else 0. */
int gbfft_supported_length(int n);
/* Stockham radix passes used for length n: writes up to `cap` radices, returns the count (<0: unsupported). */
int gbfft_radix_plan(int n, int* radices, int cap);
/* Library version string. */
const char* gbfft_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GBFFT_H */
