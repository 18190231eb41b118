// Internal types shared by the host plan code and the kernel translation units.
// Not part of the public C ABI (include/gbfft.h is).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gbfft {

// Pencils per tile. A tile is 16 pencils x the transform length; on the
// strided ("column") side of a stage the 16 pencils are 16 consecutive complex
// values = one 128-byte line per transform index.
constexpr int kTileP = 16;

enum AccessMode : int {
  kRow = 0,  // the transform axis is contiguous (element stride 1)
  kCol = 1,  // the 16 pencils of a tile are contiguous (pencil stride 1)
};

enum TileKind : int {
  kPlain = 0,     // complex transform of length L
  kR2CPost = 1,   // length-L complex FFT of real pairs, then split into L+1 bins
  kC2RPre = 2,    // merge L+1 half-spectrum bins into L complex, then FFT
  kIdentity = 3,  // no arithmetic: pure pack/transpose/unpack (debug, bit-exact tests)
  kPoissonZ = 4,  // forward FFT, multiply by -1/|k|^2, inverse FFT (fused Poisson z stage)
  kPoissonZB = 5, // bounded z: DCT-II, multiply by -1/|k|^2, DCT-III (fused Poisson z stage, Neumann walls)
  kDct2 = 6,      // real-to-real along the stage's axis: DCT-II (REDFT10) of every pencil
  kDct3 = 7,      // DCT-III (REDFT01)
  kDst2 = 8,      // DST-II (RODFT10)
  kDst3 = 9,      // DST-III (RODFT01)
};

// Arithmetic of a stage's radix-16 passes: FP32 on the CUDA cores, or dense
// 16x16 DFT products on the tensor cores with operands split into hi/lo pairs
// of FP16 or BF16 (FP32 accumulation). Storage is complex64 in every mode.
// The split modes run on the warp-level tensor-core path (mma.sync) or, for
// lengths whose radix-16 butterflies fill 128-row operand tiles, on the
// fifth-generation tensor cores (tcgen05.mma, accumulators in tensor memory).
enum StagePrec : int {
  kPrecFP32 = 0,
  kPrecF16Split = 1,
  kPrecBF16Split = 2,
  kPrecF16SplitTC5 = 3,
  kPrecBF16SplitTC5 = 4,
};

__host__ __device__ constexpr bool prec_is_tc5(int p) { return p == kPrecF16SplitTC5 || p == kPrecBF16SplitTC5; }
// the warp-level split mode with the same 16-bit operand type
__host__ __device__ constexpr int prec_mma_sync(int p) {
  return p == kPrecF16SplitTC5 ? kPrecF16Split : (p == kPrecBF16SplitTC5 ? kPrecBF16Split : p);
}

// Dependency rule of a tile on the previous stage of the same launch
// (persistent kernel only). See DepRule handling in the persistent kernel.
enum DepRule : int {
  kDepNone = 0,
  kDepGroup = 1,       // group range [g0, g0+valid) <-> producer outer ids
  kDepOuter = 2,       // outer id o <-> producer outer id o
  kDepGchunkOfOuter = 3,  // outer id o <-> producer group chunk o/16
  kDepSameGchunk = 4,  // own group chunk <-> producer group chunk
  kDepAll = 5,         // every producer tile of the same batch entry
};

// One stage of the staged 3D FFT: a batched 1D transform over pencils,
// reading one layout and writing another (the pack/transpose/unpack of the
// redistribution is the load and store of the tile).
//
// Tile t decodes as t = (b * n_outer + o) * n_gchunks + gc. Element n of
// pencil p of the tile is read at
//   in  + b*in_b  + o*in_o  + (16*gc + p)*in_g  + n*in_n
// and output element k written at
//   out + b*out_b + o*out_o + (16*gc + p)*out_g + k*out_n      (float2 units).
struct StageDesc {
  const float2* in;
  float2* out;
  long long in_b, in_o, in_g, in_n;
  long long out_b, out_o, out_g, out_n;
  long long n_tiles;
  int batch, n_outer, n_group, n_gchunks;
  int L;         // complex transform length of the pencil
  int n_in;      // elements read per pencil (L, or L+1 for kC2RPre)
  int n_out;     // elements written per pencil (L, or L+1 for kR2CPost)
  int in_mode, out_mode, kind;
  int dir;       // -1 forward sign, +1 inverse sign
  float scale;     // multiplies every output value
  float interior;  // R2C/C2R: multiplies bins 1..L-1 of the half spectrum
  const float2* tw;    // packed per-pass twiddles of length L (tw_table_len(L) entries, device)
  const float2* tw2;   // W_2L^k = exp(-2 pi i k / 2L), k in [0, L] (R2C/C2R); W_4L^k, k <= L (DCT / DST kinds)
  int tw_len;          // entries of tw
  const float2* twn;   // natural twiddles W_L^m = exp(-2 pi i m / L), m in [0, L) (device)
  // Poisson z stage: wavenumber bookkeeping of the tile's pencils
  int pz_nx, pz_ny;    // full grid nx, ny (kx of pencil = group index, ky = outer index)
  // persistent-kernel dependency rule on the previous stage
  int dep_rule;
  int prev_n_outer, prev_n_gchunks;
  int prec;  // StagePrec of the radix-16 passes (kPlain stages of staged launches)
  int body;  // persistent launches: 1 = this stage's tiles run the warp-per-pencil body (length 512), 0 = Stockham
  // Merged pencil index (warp-per-pencil launches only; 0 = off): the outer
  // and group indices run as one group index m = o * m_split + g, and the
  // row side addresses pencil m at (m / m_split) * split_o + (m % m_split) * split_g.
  int m_split;
  long long split_o, split_g;
  // device error word of the plan (kernels with bounded waits record kDevErrTimeout here); may be null
  int* err;
};

// Control block of one persistent launch (device memory, zeroed before each launch).
// The first two words persist across launches until read; a persistent
// launch clears `ticket`, `abort` and the counters that follow the struct.
struct Control {
  int error;         // first device-side error code (0 = none)
  int pad;
  unsigned int ticket;
  int abort;         // set with the error so other CTAs stop taking tickets
};

constexpr int kMaxStages = 5;

// Error codes written into Control::error by device code.
constexpr int kDevErrTimeout = 1;

}  // namespace gbfft
