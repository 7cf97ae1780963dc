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
constexpr int kNpad = 1024;                        // 4 points x 256 threads
constexpr size_t kDescBytes = (size_t)KP_STATIC_MAX_SYSTEMS * sizeof(kp::SysDesc);
constexpr size_t kDescRegion = (kDescBytes + 255) / 256 * 256;
constexpr size_t kScratchBytes = KP_STATIC_SCRATCH_BYTES;
static_assert(kScratchBytes > kDescRegion, "scratch must hold the descriptor table");

// The shared scratch: [descriptor table][Krylov-vector workspace of the blocks].
// Every call overwrites it; calls that overlap on the GPU race on it.
static __device__ __align__(256) unsigned char kp_static_scratch[kScratchBytes];

// Descriptors travel to the table as kernel parameters, 256 per launch
// (24 KB of the 32 KB parameter space), so nothing is staged in host memory
// that a later call could overwrite before the copy runs.
constexpr int kDescPerLaunch = 256;
struct DescChunk {
  int first, count;
  kp::SysDesc d[kDescPerLaunch];
};

__global__ void upload_desc_kernel(const __grid_constant__ DescChunk c, kp::SysDesc* table) {
  for (int k = threadIdx.x; k < c.count; k += blockDim.x) table[c.first + k] = c.d[k];
}

struct DeviceSetup {
  bool done = false;
  unsigned char* scratch = nullptr;   // device address of kp_static_scratch
  size_t smem_optin = 0;
  int sms = 0;
};

std::mutex g_mu;                                  // guards g_setup
DeviceSetup g_setup[kMaxDevices];

// Once per device, with that device current: resolve the scratch symbol to
// a device address (host code only sees a host-side stand-in for it) and
// read the limits the launch shape depends on.
kp_status setup_device(int dev, DeviceSetup* out) {
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceSetup& s = g_setup[dev];
  if (!s.done) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, kp_static_scratch);
    if (e != cudaSuccess) return KP_ERR_CUDA;
    int v = 0, sms = 0;
    e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return KP_ERR_CUDA;
    s.scratch = static_cast<unsigned char*>(ptr);
    s.smem_optin = (size_t)v;
    s.sms = sms;
    s.done = true;
  }
  *out = s;
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
  DeviceSetup ds;
  kp_status st = setup_device(dev, &ds);
  if (st != KP_OK) return st;
  // Shared-memory window: as many Krylov vectors as one block per SM allows;
  // the rest go to each block's slice of the static workspace.
  const size_t fixed = kp::gmres_fp64_smem_bytes(4, 256, 0, m);
  const size_t per = (size_t)kNpad * sizeof(double);
  if (ds.smem_optin <= fixed + per) return KP_ERR_UNSUPPORTED;
  const int S = (int)std::min<size_t>((size_t)m + 1, (ds.smem_optin - fixed) / per);
  // Persistent blocks, one per SM of this device, fewer if their Krylov
  // spill would not fit the array; each block marches systems k, k + grid, ...
  const size_t spill_per_block = (size_t)(m + 1 - S) * per;
  const size_t room = kScratchBytes - kDescRegion;
  const size_t fit = spill_per_block ? room / spill_per_block : (size_t)nsys;
  if (fit < 1) return KP_ERR_TOO_LARGE;
  const int grid = (int)std::min<size_t>({(size_t)nsys, (size_t)std::max(ds.sms, 1), fit});
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  kp::SysDesc* ddesc = reinterpret_cast<kp::SysDesc*>(ds.scratch);
  DescChunk chunk;
  for (int k0 = 0; k0 < nsys; k0 += kDescPerLaunch) {
    chunk.first = k0;
    chunk.count = std::min(kDescPerLaunch, nsys - k0);
    for (int k = 0; k < chunk.count; ++k) {
      const kp_op& o = ops[k0 + k];
      kp::SysDesc d{};
      d.mt = o.mtilde;
      d.fx = o.fx;
      d.fy = o.fy;
      d.b = b[k0 + k];
      d.x = x[k0 + k];
      d.H = o.H;
      d.W = o.W;
      d.dt = o.dt;
      d.g2 = o.g2;
      d.h = o.h;
      chunk.d[k] = d;
    }
    upload_desc_kernel<<<1, 128, 0, stream>>>(chunk, ddesc);
    if (cudaGetLastError() != cudaSuccess) return KP_ERR_CUDA;
  }
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
  p.spill = (S < m + 1) ? reinterpret_cast<double*>(ds.scratch + kDescRegion) : nullptr;
  p.info = info;
  const size_t smem = fixed + (size_t)S * per;
  const cudaError_t e = kp::launch_gmres_fp64_1k_grid(p, smem, grid, stream);
  return e == cudaSuccess ? KP_OK : KP_ERR_CUDA;
}
