// Allocation-free entry point: gbfft_exec_c2c_noalloc (see include/gbfft.h).
//
// Some callers cannot allocate device memory at the moment they need a
// transform: callers whose device memory is owned by a custom pool or
// framework allocator that forbids side allocations, and latency-critical
// loops where a cudaMalloc would synchronise the device. A gbfft_plan
// allocates twiddle tables, schedules and workspace, so those callers cannot
// create one at that point.
//
// This entry point runs the same stage kernels as the pencil C2C path
// (staged launches), with the intermediate stage buffer in a file-scope
// static __device__ array instead of plan workspace, and with twiddle tables
// for every supported length in a second static array. Both arrays exist on
// every GPU that loads the library, for as long as it stays loaded.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/gbfft.h"
#include "gbfft_kernels.cuh"

namespace gbfft {
int launch_stage_external(const StageDesc& d, cudaStream_t stream);
std::vector<float2> packed_twiddles(int L);
}

using namespace gbfft;

namespace {

// Scratch for the intermediate stage array C[kx][ky][kz]: one complex64 per
// grid point, GBFFT_NOALLOC_MAX_POINTS points (32 MiB). Shared by every call.
__device__ __align__(256) float2 g_noalloc_scratch[GBFFT_NOALLOC_MAX_POINTS];

// Packed twiddle tables (the stage kernels' layout) for every supported
// length L, one after another.
constexpr int kTwCapacity = 16384;
__device__ __align__(256) float2 g_noalloc_twiddles[kTwCapacity];

constexpr int kMaxLen = 1024;
constexpr int kMaxDevices = 64;

struct DeviceState {
  std::atomic<bool> ready{false};  // set once, with release order, after the fields below
  float2* scratch = nullptr;   // device address of g_noalloc_scratch on this device
  float2* tw = nullptr;        // device address of g_noalloc_twiddles on this device
  int tw_offset[kMaxLen + 1];  // offset of the W_L table, -1 if L unsupported
};

std::mutex g_mu;
DeviceState g_state[kMaxDevices];

// Set-up, once per device, with that device current: resolve the two arrays'
// device addresses and upload the twiddle tables (FP64 cos/sin, rounded once).
// A device that is ready is found without taking the lock. The upload is a
// synchronous copy, which a stream capture in progress on `stream` would not
// survive, so set-up is refused (nothing enqueued) while `stream` captures.
int setup_device(int dev, cudaStream_t stream, DeviceState** out) {
  DeviceState& st = g_state[dev];
  if (st.ready.load(std::memory_order_acquire)) {
    *out = &st;
    return GBFFT_OK;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(stream, &cs) != cudaSuccess) {
    cudaGetLastError();
    return GBFFT_ERR_CUDA;
  }
  if (cs != cudaStreamCaptureStatusNone) return GBFFT_ERR_SETUP_IN_CAPTURE;
  std::lock_guard<std::mutex> lk(g_mu);
  if (st.ready.load(std::memory_order_acquire)) {
    *out = &st;
    return GBFFT_OK;
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) return GBFFT_ERR_CUDA;
  st.scratch = reinterpret_cast<float2*>(p);
  p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_twiddles) != cudaSuccess) return GBFFT_ERR_CUDA;
  st.tw = reinterpret_cast<float2*>(p);
  std::vector<float2> host;
  host.reserve(kTwCapacity);
  for (int L = 0; L <= kMaxLen; ++L) {
    st.tw_offset[L] = -1;
    if (L < 2 || !gbfft_supported_length(L)) continue;
    const std::vector<float2> t = packed_twiddles(L);
    if ((int)(host.size() + t.size()) > kTwCapacity) return GBFFT_ERR_CUDA;
    st.tw_offset[L] = (int)host.size();
    host.insert(host.end(), t.begin(), t.end());
  }
  if (cudaMemcpyToSymbol(g_noalloc_twiddles, host.data(), host.size() * sizeof(float2)) != cudaSuccess)
    return GBFFT_ERR_CUDA;
  st.ready.store(true, std::memory_order_release);
  *out = &st;
  return GBFFT_OK;
}

StageDesc stage(const void* in, void* out, int L, int dir, int n_outer, int n_group, long long io, long long ig,
                long long in_, int im, long long oo, long long og, long long on_, int om, float scale,
                const float2* tw, long long vol) {
  StageDesc d;
  std::memset(&d, 0, sizeof(d));
  d.in = reinterpret_cast<const float2*>(in);
  d.out = reinterpret_cast<float2*>(out);
  d.in_b = vol;
  d.in_o = io;
  d.in_g = ig;
  d.in_n = in_;
  d.out_b = vol;
  d.out_o = oo;
  d.out_g = og;
  d.out_n = on_;
  d.batch = 1;
  d.n_outer = n_outer;
  d.n_group = n_group;
  d.n_gchunks = (n_group + kTileP - 1) / kTileP;
  d.n_tiles = (long long)n_outer * d.n_gchunks;
  d.L = L;
  d.n_in = L;
  d.n_out = L;
  d.in_mode = im;
  d.out_mode = om;
  d.kind = kPlain;
  d.dir = dir;
  d.scale = scale;
  d.interior = 1.f;
  d.tw = tw;
  d.tw_len = tw_table_len(L);
  return d;
}

// Largest float2 offset + 1 a stage reads / writes (one grid, positive strides).
long long read_end(const StageDesc& d) {
  return (long long)(d.n_outer - 1) * d.in_o + (long long)(d.n_group - 1) * d.in_g + (long long)(d.n_in - 1) * d.in_n +
         1;
}
long long write_end(const StageDesc& d) {
  return (long long)(d.n_outer - 1) * d.out_o + (long long)(d.n_group - 1) * d.out_g +
         (long long)(d.n_out - 1) * d.out_n + 1;
}

}  // namespace

extern "C" int gbfft_exec_c2c_noalloc(int nx, int ny, int nz, int op, const void* in, void* out, void* stream) {
  if (nx < 2 || ny < 2 || nz < 2) return GBFFT_ERR_INVALID_ARG;
  if (op < GBFFT_OP_FORWARD || op > GBFFT_OP_INVERSE_ADJOINT) return GBFFT_ERR_INVALID_ARG;
  if (!in || !out) return GBFFT_ERR_INVALID_ARG;
  if (in == out) return GBFFT_ERR_INPLACE;
  if (((uintptr_t)in) % 16 != 0 || ((uintptr_t)out) % 16 != 0) return GBFFT_ERR_ALIGNMENT;
  const long long n = (long long)nx * ny * nz;
  if (n > (long long)GBFFT_NOALLOC_MAX_POINTS) return GBFFT_ERR_STATIC_LIMIT;
  if (nx > kMaxLen || ny > kMaxLen || nz > kMaxLen || !gbfft_supported_length(nx) || !gbfft_supported_length(ny) ||
      !gbfft_supported_length(nz))
    return GBFFT_ERR_UNSUPPORTED_SIZE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GBFFT_ERR_NO_DEVICE;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  DeviceState* st = nullptr;
  int rc = setup_device(dev, s, &st);
  if (rc) return rc;
  const float2* twx = st->tw + st->tw_offset[nx];
  const float2* twy = st->tw + st->tw_offset[ny];
  const float2* twz = st->tw + st->tw_offset[nz];
  float2* W = st->scratch;
  const float invN = (float)(1.0 / (double)n);
  // Layouts: A natural [z][y][x]; B [z][x][y]; C [x][y][z]. Every element of
  // the scratch is written by one stage before the next stage reads it, so
  // nothing in it has to start at zero.
  StageDesc st3[3];
  if (op == GBFFT_OP_FORWARD || op == GBFFT_OP_INVERSE_ADJOINT) {
    const float sc = op == GBFFT_OP_INVERSE_ADJOINT ? invN : 1.f;
    st3[0] = stage(in, out, nx, -1, nz, ny, (long long)nx * ny, nx, 1, kRow, (long long)nx * ny, 1, ny, kCol, 1.f,
                   twx, n);
    st3[1] = stage(out, W, ny, -1, nx, nz, ny, (long long)nx * ny, 1, kRow, (long long)ny * nz, 1, nz, kCol, 1.f,
                   twy, n);
    st3[2] = stage(W, out, nz, -1, ny, nx, nz, (long long)ny * nz, 1, kRow, nx, 1, (long long)nx * ny, kCol, sc, twz,
                   n);
  } else {
    const float sc = op == GBFFT_OP_INVERSE ? invN : 1.f;
    st3[0] = stage(in, out, nz, +1, ny, nx, nx, 1, (long long)nx * ny, kCol, nz, (long long)ny * nz, 1, kRow, 1.f,
                   twz, n);
    st3[1] = stage(out, W, ny, +1, nx, nz, (long long)ny * nz, 1, nz, kCol, ny, (long long)nx * ny, 1, kRow, 1.f,
                   twy, n);
    st3[2] = stage(W, out, nx, +1, nz, ny, (long long)nx * ny, 1, ny, kCol, (long long)nx * ny, nx, 1, kRow, sc, twx,
                   n);
  }
  // Host-side bounds check before anything is launched: in, out and the
  // scratch each hold n points (the scratch more), so every stage's largest
  // read and write offset must stay below n.
  for (int k = 0; k < 3; ++k)
    if (read_end(st3[k]) > n || write_end(st3[k]) > n) return GBFFT_ERR_INVALID_ARG;
  for (int k = 0; k < 3; ++k) {
    rc = launch_stage_external(st3[k], s);
    if (rc) return rc;
  }
  return GBFFT_OK;
}
