// fam_noalloc.cu -- one 1D FAM time step that allocates no device memory.
//
// Some callers cannot allocate GPU memory: host applications that own a
// fixed device-memory budget and do not let plug-ins call cudaMalloc, and
// latency-critical loops where an allocation's cost and failure mode are not
// acceptable.  fam_step1d_noalloc() serves them: the caller passes the input
// and output states in device memory, and every intermediate buffer of the
// step (the padded stage states and the device control block) lives in one
// file-scope static device array of fixed size.  That array exists once per
// GPU that loads the library and stays allocated until the process exits.
//
// Host code must not use the array's name as a device address (in host code
// it names a host-side stand-in); the device address is obtained once per
// device with cudaGetSymbolAddress, with that device current, on the first
// call made on that device -- so the first call on a device should come
// before any stream capture.  Every call shares the array and overwrites it:
// calls whose GPU work overlaps (different streams, or different host
// threads) race on it and must be serialised by the caller.  Each call
// starts the control block from zero with a one-thread kernel and, at the
// end, waits for its stream and reads the control block back to report the
// step size and the device flags.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "fam_internal.cuh"

namespace {

constexpr int kMaxCells = FAM_NOALLOC_MAX_CELLS;
constexpr int kMaxPlanes = 6;                                    // 1D Euler: 3 components x 2 moments
constexpr long long kPitchMax = ((kMaxCells + 2 * G) + 31) / 32 * 32;  // >= any pitch used
constexpr size_t kCtlBytes = 512;                                // FamCtl, padded to the alignment
constexpr size_t kBufBytes = sizeof(double) * (size_t)kMaxPlanes * (size_t)kPitchMax;
constexpr size_t kScratchBytes = kCtlBytes + 3 * kBufBytes;
static_assert(sizeof(FamCtl) <= kCtlBytes, "control block must fit its slot");
static_assert(kBufBytes % 256 == 0, "buffers start 256-byte aligned");

// The scratch: control block, then the three padded state buffers.
static __device__ __align__(256) unsigned char g_fam_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set-up once).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_fam_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

// Start the control block of a call from `init` (passed by value: no host
// buffer has to outlive the launch).
__global__ void noalloc_ctl_reset(FamCtl* ctl, const FamCtl init) { *ctl = init; }

}  // namespace

// defined in fam_api.cu
fam_status fam_internal_encode_maps(fam_handle* h);
fam_status fam_internal_fill_ghosts(fam_handle* h, int b);
bool fam_internal_pick(fam_handle* h);

extern "C" fam_status fam_step1d_noalloc(const void* U_in, void* U_out, int nx, double x0, double x1, int k,
                                         int equation, int bc, double gamma, int precision, double cfl,
                                         double* dt_used, void* stream) {
  if (!U_in || !U_out) return FAM_E_INVAL;
  if (nx < 4 || nx > kMaxCells) return FAM_E_INVAL;  // beyond the static scratch
  if (k < 3 || k > 6 || !(x1 > x0) || !(cfl > 0.0)) return FAM_E_INVAL;
  if (equation < FAM_ADVECTION || equation > FAM_EULER) return FAM_E_INVAL;
  if (bc != FAM_BC_PERIODIC && bc != FAM_BC_OUTFLOW) return FAM_E_INVAL;
  if (precision != 64 && precision != 32) return FAM_E_INVAL;
  if (equation == FAM_EULER && !(gamma > 1.0)) return FAM_E_INVAL;

  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return FAM_E_CUDA;

  // a handle on the host stack whose buffers are slices of the scratch
  fam_handle h;
  h.d = 1;
  h.k = k;
  h.eq = equation;
  h.bc = bc;
  h.prec = precision;
  h.gamma = gamma;
  h.ax = h.ay = equation == FAM_ADVECTION ? gamma : 1.0;
  h.nc = equation == FAM_EULER ? 3 : 1;
  h.nm = 2;
  h.np = h.nc * 2;
  h.elem = precision == 64 ? 8 : 4;
  Geo& g = h.geo;
  g.nx = nx;
  g.ny = 1;
  g.px = ((nx + 2 * G) + 3) / 4 * 4;
  g.rows = 1;
  g.plane = g.px;
  g.bcx = g.bcy = bc;
  for (int q = 0; q < 4; ++q) g.bc[q] = bc;
  g.nm = 2;
  g.euler = equation == FAM_EULER;
  g.dx = (x1 - x0) / nx;
  g.dy = 1.0;
  g.idx = 1.0 / g.dx;
  g.idy = 1.0;
  h.stream = reinterpret_cast<cudaStream_t>(stream);
  h.own_stream = false;
  unsigned char* p = reinterpret_cast<unsigned char*>(base);
  h.ctl = reinterpret_cast<FamCtl*>(p);
  for (int b = 0; b < 3; ++b) h.buf[b] = p + kCtlBytes + (size_t)b * kBufBytes;
  if (!fam_internal_pick(&h)) return FAM_E_UNSUPPORTED;
  if (h.ops.prepare() != cudaSuccess) return FAM_E_CUDA;
  if (fam_internal_encode_maps(&h) != FAM_OK) return FAM_E_CUDA;

  // the control block keeps the previous call's contents: start it from zero
  FamCtl c;
  std::memset(&c, 0, sizeof(c));
  c.cfl = cfl;
  c.dim = 1;
  c.dx = g.dx;
  c.dy = 1.0;
  c.dxe = g.dx;
  c.dye = 1.0;
  noalloc_ctl_reset<<<1, 1, 0, h.stream>>>(h.ctl, c);
  if (cudaGetLastError() != cudaSuccess) return FAM_E_CUDA;
  // input -> padded buffer A (+ ghost images)
  const size_t row = (size_t)nx * h.elem;
  for (int q = 0; q < h.np; ++q) {
    char* d0 = reinterpret_cast<char*>(h.buf[0]) + ((size_t)q * g.plane + G) * h.elem;
    const char* s0 = reinterpret_cast<const char*>(U_in) + (size_t)q * row;
    if (cudaMemcpyAsync(d0, s0, row, cudaMemcpyDeviceToDevice, h.stream) != cudaSuccess) return FAM_E_CUDA;
  }
  if (fam_internal_fill_ghosts(&h, 0) != FAM_OK) return FAM_E_CUDA;
  // step size from the averages, then the three stages and the OE
  if (h.ops.alpha(&h, 0) != cudaSuccess) return FAM_E_CUDA;
  if (h.ops.stage(&h, 0, 0, 1, 1) != cudaSuccess) return FAM_E_CUDA;
  if (h.ops.stage(&h, 1, 0, 2, 2) != cudaSuccess) return FAM_E_CUDA;
  if (h.ops.stage(&h, 2, 0, 1, 3) != cudaSuccess) return FAM_E_CUDA;
  if (h.ops.oe(&h, 1, 0, -1.0) != cudaSuccess) return FAM_E_CUDA;
  for (int q = 0; q < h.np; ++q) {
    const char* s0 = reinterpret_cast<const char*>(h.buf[0]) + ((size_t)q * g.plane + G) * h.elem;
    char* d0 = reinterpret_cast<char*>(U_out) + (size_t)q * row;
    if (cudaMemcpyAsync(d0, s0, row, cudaMemcpyDeviceToDevice, h.stream) != cudaSuccess) return FAM_E_CUDA;
  }
  // Every call waits for its step and reads the device flags, so that a
  // non-physical or timed-out step is never reported as FAM_OK.  The step
  // size taken is the one the OE epilogue advanced the clock by.
  FamCtl out;
  if (cudaMemcpyAsync(&out, h.ctl, sizeof(out), cudaMemcpyDeviceToHost, h.stream) != cudaSuccess) return FAM_E_CUDA;
  if (cudaStreamSynchronize(h.stream) != cudaSuccess) return FAM_E_CUDA;
  if (dt_used) *dt_used = out.t;
  if (out.status & kStatusTimeout) return FAM_E_TIMEOUT;
  if (out.status & (kStatusNonFinite | kStatusNonPhysical)) return FAM_E_NONPHYSICAL;
  return FAM_OK;
}
