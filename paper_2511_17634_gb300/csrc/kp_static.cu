// kp_static.cu -- kp_refine_static: the refine GMRES of kp_refine for callers
// that cannot allocate device memory.
//
// Some callers may not call cudaMalloc (or any allocating routine) at the
// point where they need a solve: code running while a memory pool or arena
// owns the device memory, plugins whose host forbids allocation after
// start-up, or latency-critical paths that must never reach the allocator.
// kp_refine needs a context (kp_create allocates the basis store) and grows
// device workspaces on demand, so it cannot serve them.  This entry point
// needs no context: its scratch -- the per-call system descriptors and the
// Krylov vectors that do not fit in shared memory -- lives in one file-scope
// device array that exists from the moment the library's module is loaded
// onto a GPU until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "kp.h"
#include "kp_internal.cuh"

namespace {

constexpr int kMaxDevices = 64;
constexpr int kGrid = KP_STATIC_BLOCKS;           // thread blocks per call (persistent)
constexpr int kNpad = 1024;                        // 4 points x 256 threads
constexpr size_t kDescBytes = (size_t)KP_STATIC_MAX_SYSTEMS * sizeof(kp::SysDesc);
constexpr size_t kDescRegion = (kDescBytes + 255) / 256 * 256;
constexpr size_t kScratchBytes = KP_STATIC_SCRATCH_BYTES;
static_assert(kScratchBytes > kDescRegion, "scratch must hold the descriptor table");

// The shared scratch: [descriptor table][Krylov-vector workspace of kGrid blocks].
// Every call overwrites it; calls that overlap on the GPU race on it.
static __device__ __align__(256) unsigned char kp_static_scratch[kScratchBytes];

struct DeviceSetup {
  bool done = false;
  unsigned char* scratch = nullptr;   // device address of kp_static_scratch
  size_t smem_optin = 0;
};

std::mutex g_mu;                                  // guards g_setup and g_host_desc
DeviceSetup g_setup[kMaxDevices];
kp::SysDesc g_host_desc[KP_STATIC_MAX_SYSTEMS];   // host staging of the descriptors

// Once per device, with that device current: resolve the scratch symbol to
// a device address (host code only sees a host-side stand-in for it).
kp_status setup_device(int dev, DeviceSetup** out) {
  DeviceSetup& s = g_setup[dev];
  if (!s.done) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, kp_static_scratch);
    if (e != cudaSuccess) return KP_ERR_CUDA;
    int v = 0;
    e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return KP_ERR_CUDA;
    s.scratch = static_cast<unsigned char*>(ptr);
    s.smem_optin = (size_t)v;
    s.done = true;
  }
  *out = &s;
  return KP_OK;
}

}  // namespace

extern "C" kp_status kp_refine_static(int nsys, const kp_op* ops, const double* const* b,
                                      double* const* x, double tol, int m, int maxit,
                                      kp_info* info, void* cuda_stream) {
  if (nsys < 0 || m < 1 || m > kp::kMaxM || maxit < 0 || !(tol >= 0.0)) return KP_ERR_ARG;
  if (nsys == 0) return KP_OK;
  if (!ops || !b || !x) return KP_ERR_ARG;
  if (nsys > KP_STATIC_MAX_SYSTEMS) return KP_ERR_TOO_LARGE;
  for (int k = 0; k < nsys; ++k) {
    const kp_op& o = ops[k];
    if (o.H < 1 || o.W < 1 || !o.mtilde || !b[k] || !x[k]) return KP_ERR_ARG;
    if ((long long)o.H * o.W > KP_STATIC_MAX_N) return KP_ERR_TOO_LARGE;
    if (!(o.dt > 0.0) || !(o.h > 0.0) || !(o.g2 >= 0.0)) return KP_ERR_ARG;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return KP_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return KP_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceSetup* ds = nullptr;
  kp_status st = setup_device(dev, &ds);
  if (st != KP_OK) return st;
  // Shared-memory window: as many Krylov vectors as one block per SM allows;
  // the rest go to this call's slice of the static workspace.
  const size_t fixed = kp::gmres_fp64_smem_bytes(4, 256, 0, m);
  const size_t per = (size_t)kNpad * sizeof(double);
  if (ds->smem_optin <= fixed + per) return KP_ERR_UNSUPPORTED;
  const int S = (int)std::min<size_t>((size_t)m + 1, (ds->smem_optin - fixed) / per);
  const int grid = std::min(nsys, kGrid);
  const size_t spill_bytes = (size_t)grid * (size_t)(m + 1 - S) * per;
  if (kDescRegion + spill_bytes > kScratchBytes) return KP_ERR_TOO_LARGE;
  for (int k = 0; k < nsys; ++k) {
    kp::SysDesc d{};
    d.mt = ops[k].mtilde;
    d.fx = ops[k].fx;
    d.fy = ops[k].fy;
    d.b = b[k];
    d.x = x[k];
    d.H = ops[k].H;
    d.W = ops[k].W;
    d.dt = ops[k].dt;
    d.g2 = ops[k].g2;
    d.h = ops[k].h;
    g_host_desc[k] = d;
  }
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  kp::SysDesc* ddesc = reinterpret_cast<kp::SysDesc*>(ds->scratch);
  // pageable source: the call returns once the bytes are staged, so the host
  // table can be reused by the next call
  cudaError_t e = cudaMemcpyAsync(ddesc, g_host_desc, (size_t)nsys * sizeof(kp::SysDesc),
                                  cudaMemcpyHostToDevice, stream);
  if (e != cudaSuccess) return KP_ERR_CUDA;
  kp::GmresParams p{};
  p.sys = ddesc;
  p.nsys = nsys;
  p.tol = tol;
  p.m = m;
  p.maxit = maxit;
  p.S = S;
  p.reorth = 0;
  p.npad = kNpad;
  p.b_scale = 1.0;
  p.x0_mode = kp::X0_READ;
  p.spill = (S < m + 1) ? reinterpret_cast<double*>(ds->scratch + kDescRegion) : nullptr;
  p.info = info;
  const size_t smem = fixed + (size_t)S * per;
  e = kp::launch_gmres_fp64_1k_grid(p, smem, grid, stream);
  return e == cudaSuccess ? KP_OK : KP_ERR_CUDA;
}
