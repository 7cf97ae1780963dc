// kp_api.cu -- the C ABI declared in include/kp.h: context, argument checks,
// descriptor upload and kernel launches.  No compute happens on the host.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kp.h"
#include "kp_ctx.h"
#include "kp_internal.cuh"

using kp::CapMeta;
using kp::SlotMeta;
using kp::SysDesc;

namespace kp {

kp_status set_error(kp_ctx* c, kp_status s, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return s;
}

kp_status cuda_error(kp_ctx* c, cudaError_t e, const char* what) {
  return set_error(c, e == cudaErrorMemoryAllocation ? KP_ERR_OOM : KP_ERR_CUDA, "%s: %s", what,
                   cudaGetErrorString(e));
}

cudaError_t launch_solver(const GmresParams& p, const Shape& sh, bool mixed, cudaStream_t st) {
  if (sh.cs > 0) return launch_gmres_cluster(p, sh.ept, sh.nt, sh.cs, sh.minb, sh.smem, st);
  return mixed ? launch_gmres_mixed(p, sh.ept, sh.nt, sh.smem, st)
               : launch_gmres_fp64(p, sh.ept, sh.nt, sh.minb, sh.smem, st);
}

kp_status gmres_shape(kp_ctx* c, int nmax, int m, Shape* out, bool mixed, int wmin) {
  Shape sh;
  sh.minb = 1;
  if (nmax <= 1024) {
    // default (FP64): 128 threads x 8 points, 4 resident blocks per SM -- more
    // independent systems per SM hide the per-step barriers and the serial
    // Givens work better than 256 x 4 at 2 blocks (measured: 4.0 vs 3.3 M
    // systems/s on the 32x32x3 march)
    sh.nt = c->opt.block_threads ? c->opt.block_threads : (mixed ? 256 : 128);
    sh.ept = 1024 / sh.nt;
    sh.minb = c->opt.blocks_per_sm ? c->opt.blocks_per_sm : (sh.nt == 128 && !c->opt.block_threads ? 4
                                                             : sh.nt == 64 ? 4 : 2);
    if (mixed) {                                 // the FP32 solver has the 2-block 256/128 shapes
      sh.minb = 2;
      if (sh.nt == 64) { sh.nt = 128; sh.ept = 8; }
    }
  }
  else if (nmax <= 4096 && !(mixed && c->opt.cluster_size)) { sh.ept = 8; sh.nt = 512; }
  else if (mixed) {
    // a cluster of cs CTAs, each holding W/cs whole columns (<= 2048 points;
    // 16-CTA clusters: 128 threads and <= 1024 points per CTA)
    sh.ept = 8; sh.nt = c->opt.cluster_size == 16 ? 128 : 256;
    if (c->opt.cluster_size) {
      if ((nmax + c->opt.cluster_size - 1) / c->opt.cluster_size <= sh.ept * sh.nt) sh.cs = c->opt.cluster_size;
    } else {
      for (int cs : {2, 4, 8})
        if ((nmax + cs - 1) / cs <= 2048) { sh.cs = cs; break; }
    }
    if (!sh.cs || wmin <= 0 || wmin % sh.cs)
      return set_error(c, KP_ERR_UNSUPPORTED, "N=%d: needs W divisible by the cluster size and N <= 16384", nmax);
    sh.minb = c->opt.cluster_blocks_per_sm ? c->opt.cluster_blocks_per_sm : (sh.cs == 16 ? 4 : 2);
    if (sh.cs == 16 ? (sh.minb != 2 && sh.minb != 4) : sh.minb > 2)
      return set_error(c, KP_ERR_UNSUPPORTED, "cluster of %d CTAs: %d CTAs per SM not built", sh.cs, sh.minb);
  }
  else return set_error(c, KP_ERR_UNSUPPORTED, "N=%d: FP64 grids above 4096 unknowns are not supported (use the mixed-precision mode)", nmax);
  const int npad = sh.ept * sh.nt;
  const size_t fixed = sh.cs ? gmres_cluster_smem_bytes(sh.ept, sh.nt, 0, m)
                     : mixed ? gmres_mixed_smem_bytes(sh.ept, sh.nt, 0, m)
                             : gmres_fp64_smem_bytes(sh.ept, sh.nt, 0, m);
  const size_t per = (size_t)npad * (mixed ? sizeof(float) : sizeof(double));
  int S = c->opt.smem_vectors;
  if (S <= 0) {
    // small systems: leave room for minb resident blocks per SM (1 KB of
    // shared memory per block is reserved by the hardware)
    // (clusters: every CTA of a system's cluster sits on its own SM, and MINB
    // systems' CTAs share one)
    const size_t budget = sh.cs ? c->smem_optin / sh.minb - (sh.minb >= 2 ? 1024 : 0)
                        : npad <= 1024 ? c->smem_optin / sh.minb - (sh.minb > 2 ? 1024 : 0)
                                       : c->smem_optin;
    S = budget > fixed ? (int)((budget - fixed) / per) : 0;
  }
  S = std::min(S, m + 1);
  while (S > 1 && fixed + S * per > c->smem_optin) --S;
  if (S < 1) return set_error(c, KP_ERR_UNSUPPORTED, "shared memory too small");
  sh.S = S;
  sh.smem = fixed + S * per;
  *out = sh;
  return KP_OK;
}

}  // namespace kp

namespace {

template <typename T>
cudaError_t grow(T** p, size_t* cap_bytes, size_t need_bytes) {
  if (*cap_bytes >= need_bytes) return cudaSuccess;
  if (*p) {
    cudaError_t e = cudaFree(*p);   // synchronises the device: no kernel still reads *p
    if (e != cudaSuccess) return e;
    *p = nullptr;
  }
  *cap_bytes = 0;
  cudaError_t e = cudaMalloc((void**)p, need_bytes);
  if (e == cudaSuccess) *cap_bytes = need_bytes;
  return e;
}

// Validate the operator descriptors of a call; returns the largest N.
kp_status check_ops(kp_ctx* c, int nsys, const kp_op* ops, int* nmax) {
  if (nsys < 0) return kp::set_error(c, KP_ERR_ARG, "nsys < 0");
  if (nsys > 0 && !ops) return kp::set_error(c, KP_ERR_ARG, "ops is NULL");
  int mx = 0;
  for (int k = 0; k < nsys; ++k) {
    const kp_op& o = ops[k];
    if (o.H < 1 || o.W < 1) return kp::set_error(c, KP_ERR_ARG, "system %d: H, W must be >= 1", k);
    const long long n = (long long)o.H * o.W;
    if (n > c->opt.max_n) return kp::set_error(c, KP_ERR_ARG, "system %d: N=%lld exceeds max_n=%d", k, n, c->opt.max_n);
    if (!(o.dt > 0.0) || !(o.h > 0.0) || !(o.g2 >= 0.0))
      return kp::set_error(c, KP_ERR_ARG, "system %d: need dt > 0, h > 0, g2 >= 0", k);
    mx = std::max(mx, (int)n);
  }
  *nmax = mx;
  return KP_OK;
}

// Upload nsys descriptors through the pinned ring; returns the device copy.
kp_status upload(kp_ctx* c, const std::vector<SysDesc>& h, SysDesc** out) {
  const size_t n = h.size();
  if (n == 0) { *out = c->d_desc; return KP_OK; }
  kp::Staging& s = c->ring[c->ring_next];
  c->ring_next = (c->ring_next + 1) % kp::kRing;
  cudaError_t e;
  if (s.pending) {
    e = cudaEventSynchronize(s.done);       // the copy that last read this slot is done
    if (e != cudaSuccess) return kp::cuda_error(c, e, "cudaEventSynchronize");
    s.pending = false;
  }
  if (s.cap < n) {
    if (s.host) cudaFreeHost(s.host);
    s.host = nullptr;
    s.cap = 0;
    e = cudaMallocHost((void**)&s.host, n * sizeof(SysDesc));
    if (e != cudaSuccess) return kp::cuda_error(c, e, "cudaMallocHost");
    s.cap = n;
  }
  std::memcpy(s.host, h.data(), n * sizeof(SysDesc));
  e = grow(&c->d_desc, &c->d_desc_cap, n * sizeof(SysDesc));
  if (e != cudaSuccess) return kp::cuda_error(c, e, "cudaMalloc(descriptors)");
  e = cudaMemcpyAsync(c->d_desc, s.host, n * sizeof(SysDesc), cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return kp::cuda_error(c, e, "cudaMemcpyAsync(descriptors)");
  e = cudaEventRecord(s.done, c->stream);
  if (e != cudaSuccess) return kp::cuda_error(c, e, "cudaEventRecord");
  s.pending = true;
  *out = c->d_desc;
  return KP_OK;
}

SysDesc make_desc(const kp_op& o, const double* b, double* x, int slot) {
  SysDesc d{};
  d.mt = o.mtilde;
  d.fx = o.fx;
  d.fy = o.fy;
  d.b = b;
  d.x = x;
  d.H = o.H;
  d.W = o.W;
  d.dt = o.dt;
  d.g2 = o.g2;
  d.h = o.h;
  d.slot = slot;
  d.pad_ = 0;
  return d;
}

kp_status run_gmres(kp_ctx* c, int nsys, const kp_op* ops, const double* const* b,
                    double* const* x, double tol, int m, int maxit, kp_info* info,
                    bool capture) {
  int nmax = 0;
  kp_status st = check_ops(c, nsys, ops, &nmax);
  if (st != KP_OK) return st;
  if (m < 1 || m > kp::kMaxM) return kp::set_error(c, KP_ERR_ARG, "restart length m=%d not in [1, %d]", m, kp::kMaxM);
  if (maxit < 0) return kp::set_error(c, KP_ERR_ARG, "maxit < 0");
  if (!(tol >= 0.0)) return kp::set_error(c, KP_ERR_ARG, "tol must be >= 0");
  if (nsys == 0) return KP_OK;
  if (!b || !x) return kp::set_error(c, KP_ERR_ARG, "b or x is NULL");
  const bool mixed = c->opt.precision == KP_PREC_MIXED;
  for (int k = 0; k < nsys; ++k) {
    if (!ops[k].mtilde || !b[k] || !x[k]) return kp::set_error(c, KP_ERR_ARG, "system %d: NULL vector", k);
  }
  int wmin = 1 << 30;
  for (int k = 0; k < nsys; ++k) wmin = std::min(wmin, ops[k].W);
  for (int k = 0; k < nsys && nmax > 4096; ++k)
    if ((long long)ops[k].H * ops[k].W != nmax)
      return kp::set_error(c, KP_ERR_UNSUPPORTED, "grids above 4096 unknowns must share one size per call");
  kp::Shape sh;
  st = kp::gmres_shape(c, nmax, m, &sh, mixed, wmin);
  if (st != KP_OK) return st;
  const int ept = sh.ept, nt = sh.nt, S = sh.S, npad = ept * nt;
  const size_t smem = sh.smem;
  cudaError_t e;
  if (S < m + 1) {
    const size_t need = (size_t)nsys * (sh.cs ? sh.cs : 1) * (m + 1 - S) * npad *
                        (mixed ? sizeof(float) : sizeof(double));
    e = mixed ? grow(&c->spill32, &c->spill32_bytes, need) : grow(&c->spill, &c->spill_bytes, need);
    if (e != cudaSuccess) return kp::cuda_error(c, e, "cudaMalloc(Krylov workspace)");
  }
  if (capture) {
    const int a = c->opt.max_a;
    if (nsys > c->cap_nsys) {
      cudaFree(c->capV); cudaFree(c->capV32); cudaFree(c->capH); cudaFree(c->capMeta);
      c->capV = nullptr; c->capV32 = nullptr; c->capH = nullptr; c->capMeta = nullptr; c->cap_nsys = 0;
      if (mixed)
        e = cudaMalloc((void**)&c->capV32, (size_t)nsys * (a + 1) * c->opt.max_n * sizeof(float));
      else
        e = cudaMalloc((void**)&c->capV, (size_t)nsys * (a + 1) * c->opt.max_n * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc((void**)&c->capH, (size_t)nsys * (a + 1) * a * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc((void**)&c->capMeta, (size_t)nsys * sizeof(CapMeta));
      if (e != cudaSuccess) return kp::cuda_error(c, e, "cudaMalloc(capture)");
      c->cap_nsys = nsys;
    }
    e = cudaMemsetAsync(c->capMeta, 0, (size_t)nsys * sizeof(CapMeta), c->stream);
    if (e != cudaSuccess) return kp::cuda_error(c, e, "cudaMemsetAsync");
    c->cap_last = nsys;
  }
  std::vector<SysDesc> h(nsys);
  for (int k = 0; k < nsys; ++k) h[k] = make_desc(ops[k], b[k], x[k], 0);
  SysDesc* dd = nullptr;
  st = upload(c, h, &dd);
  if (st != KP_OK) return st;
  kp::GmresParams p{};
  p.sys = dd;
  p.nsys = nsys;
  p.tol = tol;
  p.m = m;
  p.maxit = maxit;
  p.S = S;
  p.reorth = c->opt.reorth;
  p.inner_eta = kp::inner_eta(c->opt);
  p.npad = npad;
  p.b_scale = 1.0;
  p.x0_mode = kp::X0_READ;
  p.spill = (!mixed && S < m + 1) ? c->spill : nullptr;
  p.spill32 = (mixed && S < m + 1) ? c->spill32 : nullptr;
  p.info = info;
  if (capture) {
    p.capV = c->capV;
    p.capV32 = c->capV32;
    p.capH = c->capH;
    p.capMeta = c->capMeta;
    p.cap_a = c->opt.max_a;
    p.cap_ld = c->opt.max_n;
    p.fixed_a = c->opt.fixed_a;
  }
  (void)ept; (void)nt; (void)smem;
  e = kp::launch_solver(p, sh, mixed, c->stream);
  if (e != cudaSuccess) return kp::cuda_error(c, e, "GMRES launch");
  return KP_OK;
}

}  // namespace

extern "C" {

const char* kp_version(void) { return "kp 0.1 sm_103a"; }

void kp_options_default(kp_options* o) {
  if (!o) return;
  o->max_seeds = 64;
  o->max_a = 40;
  o->max_n = 4096;
  o->precision = KP_PREC_FP64;
  o->smem_vectors = 0;
  o->reorth = 0;
  o->block_threads = 0;
  o->blocks_per_sm = 0;
  o->cluster_size = 0;
  o->fixed_a = 0;
  o->inner_digits = 0;
  o->cluster_blocks_per_sm = 0;
}

kp_status kp_create(kp_ctx** out, const kp_options* opt, void* stream) {
  if (!out) return KP_ERR_ARG;
  *out = nullptr;
  kp_options o;
  kp_options_default(&o);
  if (opt) o = *opt;
  if (o.max_seeds < 1 || o.max_a < 1 || o.max_a > kp::kMaxM || o.max_n < 1 || o.max_n > 16384 ||
      (o.precision != KP_PREC_FP64 && o.precision != KP_PREC_MIXED) ||
      o.smem_vectors < 0 || (o.reorth != 0 && o.reorth != 1) ||
      (o.block_threads != 0 && o.block_threads != 64 && o.block_threads != 128 && o.block_threads != 256) ||
      (o.cluster_size != 0 && o.cluster_size != 2 && o.cluster_size != 4 && o.cluster_size != 8 &&
       o.cluster_size != 16) ||
      (o.fixed_a != 0 && o.fixed_a != 1) || o.inner_digits < 0 || o.inner_digits > 7 ||
      o.cluster_blocks_per_sm < 0 || o.cluster_blocks_per_sm > 4)
    return KP_ERR_ARG;
  {
    // solver shapes compiled for grids of <= 1024 points: (threads, blocks per SM)
    const int bt = o.block_threads ? o.block_threads : 128;
    const int mb = o.blocks_per_sm ? o.blocks_per_sm : (!o.block_threads || bt == 64 ? 4 : 2);
    const bool ok = (bt == 256 && (mb == 2 || mb == 3)) || (bt == 128 && mb >= 2 && mb <= 4) ||
                    (bt == 64 && mb == 4);
    if (!ok || o.blocks_per_sm < 0) return KP_ERR_ARG;
  }
  kp_ctx* c = new (std::nothrow) kp_ctx();
  if (!c) return KP_ERR_OOM;
  c->opt = o;
  c->stream = (cudaStream_t)stream;
  cudaError_t e = cudaGetDevice(&c->device);
  int v = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
  c->smem_optin = (size_t)v;
  for (int i = 0; i < kp::kRing && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&c->ring[i].done, cudaEventDisableTiming);
  const size_t a = o.max_a;
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->slotV, (size_t)o.max_seeds * (a + 1) * o.max_n * sizeof(double));
  if (e == cudaSuccess && o.precision == KP_PREC_MIXED)
    e = cudaMalloc((void**)&c->slotV32, (size_t)o.max_seeds * (a + 1) * o.max_n * sizeof(float));
  if (e == cudaSuccess && o.precision == KP_PREC_MIXED) {
    c->vb_ld = (o.max_n + 7) / 8 * 8;
    e = cudaMalloc((void**)&c->slotVb, (size_t)o.max_seeds * kp::kVbRows * c->vb_ld * sizeof(__nv_bfloat16));
    if (e == cudaSuccess)   // rows past a basis are read by the GEMM: keep them finite
      e = cudaMemset(c->slotVb, 0, (size_t)o.max_seeds * kp::kVbRows * c->vb_ld * sizeof(__nv_bfloat16));
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->slotMeta, (size_t)o.max_seeds * sizeof(SlotMeta));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->slotR, (size_t)o.max_seeds * (a + 1) * a * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->slotRot, (size_t)o.max_seeds * 3 * a * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&c->slotH, (size_t)o.max_seeds * (a + 1) * a * sizeof(double));
  if (e == cudaSuccess) {
    std::vector<SlotMeta> init(o.max_seeds);
    for (auto& s : init) { std::memset(&s, 0, sizeof(s)); s.timestep = -1; }
    e = cudaMemcpy(c->slotMeta, init.data(), init.size() * sizeof(SlotMeta), cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    kp_status s = (e == cudaErrorMemoryAllocation) ? KP_ERR_OOM : KP_ERR_CUDA;
    kp_destroy(c);
    return s;
  }
  c->slot_timestep.assign(o.max_seeds, -1);
  c->slot_n.assign(o.max_seeds, 0);
  *out = c;
  return KP_OK;
}

kp_status kp_destroy(kp_ctx* c) {
  if (!c) return KP_OK;
  cudaStreamSynchronize(c->stream);
  for (auto& s : c->ring) {
    if (s.host) cudaFreeHost(s.host);
    if (s.done) cudaEventDestroy(s.done);
  }
  cudaFree(c->d_desc);
  cudaFree(c->capV);
  cudaFree(c->capH);
  cudaFree(c->capMeta);
  cudaFree(c->slotV);
  cudaFree(c->slotV32);
  cudaFree(c->slotVb);
  cudaFree(c->capV32);
  cudaFree(c->spill32);
  cudaFree(c->slotMeta);
  cudaFree(c->slotR);
  cudaFree(c->slotRot);
  cudaFree(c->slotH);
  cudaFree(c->spill);
  cudaFree(c->d_tiles);
  cudaFree(c->d_err);
  delete c;
  return KP_OK;
}

kp_status kp_set_stream(kp_ctx* c, void* stream) {
  if (!c) return KP_ERR_ARG;
  c->stream = (cudaStream_t)stream;
  return KP_OK;
}

const char* kp_last_error(kp_ctx* c) { return c ? c->err : "NULL context"; }

kp_status kp_apply(kp_ctx* c, int nsys, const kp_op* ops, const double* const* x, double* const* y) {
  if (!c) return KP_ERR_ARG;
  int nmax = 0;
  kp_status st = check_ops(c, nsys, ops, &nmax);
  if (st != KP_OK) return st;
  if (nsys == 0) return KP_OK;
  if (!x || !y) return kp::set_error(c, KP_ERR_ARG, "x or y is NULL");
  std::vector<SysDesc> h(nsys);
  for (int k = 0; k < nsys; ++k) {
    if (!ops[k].mtilde || !x[k] || !y[k]) return kp::set_error(c, KP_ERR_ARG, "system %d: NULL vector", k);
    h[k] = make_desc(ops[k], x[k], y[k], 0);
  }
  SysDesc* dd;
  st = upload(c, h, &dd);
  if (st != KP_OK) return st;
  cudaError_t e = kp::launch_apply(dd, nsys, 0, c->stream);
  return e == cudaSuccess ? KP_OK : kp::cuda_error(c, e, "apply launch");
}

kp_status kp_rhs(kp_ctx* c, int nsys, const kp_op* ops, const double* const* mprev, double* const* b) {
  if (!c) return KP_ERR_ARG;
  int nmax = 0;
  kp_status st = check_ops(c, nsys, ops, &nmax);
  if (st != KP_OK) return st;
  if (nsys == 0) return KP_OK;
  if (!mprev || !b) return kp::set_error(c, KP_ERR_ARG, "mprev or b is NULL");
  std::vector<SysDesc> h(nsys);
  for (int k = 0; k < nsys; ++k) {
    if (!mprev[k] || !b[k]) return kp::set_error(c, KP_ERR_ARG, "system %d: NULL vector", k);
    h[k] = make_desc(ops[k], mprev[k], b[k], 0);
  }
  SysDesc* dd;
  st = upload(c, h, &dd);
  if (st != KP_OK) return st;
  cudaError_t e = kp::launch_apply(dd, nsys, 1, c->stream);
  return e == cudaSuccess ? KP_OK : kp::cuda_error(c, e, "rhs launch");
}

kp_status kp_residual(kp_ctx* c, int nsys, const kp_op* ops, const double* const* b,
                      const double* const* x, double* const* r) {
  if (!c) return KP_ERR_ARG;
  if (!b || !x || !r) return nsys ? kp::set_error(c, KP_ERR_ARG, "b, x or r is NULL") : KP_OK;
  kp_status st = kp_apply(c, nsys, ops, x, r);             // r = A x
  if (st != KP_OK || nsys == 0) return st;
  std::vector<SysDesc> h(nsys);
  for (int k = 0; k < nsys; ++k) {
    if (!b[k]) return kp::set_error(c, KP_ERR_ARG, "system %d: NULL vector", k);
    h[k] = make_desc(ops[k], b[k], r[k], 0);
  }
  SysDesc* dd;
  st = upload(c, h, &dd);
  if (st != KP_OK) return st;
  cudaError_t e = kp::launch_apply(dd, nsys, 2, c->stream);    // r = b - r
  return e == cudaSuccess ? KP_OK : kp::cuda_error(c, e, "residual launch");
}

kp_status kp_seed_solve(kp_ctx* c, int nsys, const kp_op* ops, const double* const* b,
                        double* const* x, double tol, int m, int maxit, kp_info* info) {
  if (!c) return KP_ERR_ARG;
  return run_gmres(c, nsys, ops, b, x, tol, m, maxit, info, true);
}

kp_status kp_refine(kp_ctx* c, int nsys, const kp_op* ops, const double* const* b,
                    double* const* x, double tol, int m, int maxit, kp_info* info) {
  if (!c) return KP_ERR_ARG;
  return run_gmres(c, nsys, ops, b, x, tol, m, maxit, info, false);
}

kp_status kp_store_basis(kp_ctx* c, int seed_id, int timestep, int sys) {
  if (!c) return KP_ERR_ARG;
  if (seed_id < 0 || seed_id >= c->opt.max_seeds)
    return kp::set_error(c, KP_ERR_ARG, "seed_id %d not in [0, %d)", seed_id, c->opt.max_seeds);
  if (timestep < 0) return kp::set_error(c, KP_ERR_ARG, "timestep < 0");
  if (sys < 0 || sys >= c->cap_last)
    return kp::set_error(c, KP_ERR_NO_BASIS, "system %d not in the last seed solve (%d systems)", sys, c->cap_last);
  kp::FactorParams p{};
  p.capV = c->capV;
  p.capH = c->capH;
  p.capMeta = c->capMeta;
  p.sys = sys;
  p.cap_a = c->opt.max_a;
  p.cap_ld = c->opt.max_n;
  p.slotV = c->slotV;
  p.meta = c->slotMeta;
  p.slotR = c->slotR;
  p.slotRot = c->slotRot;
  p.slotH = c->slotH;
  p.seed_id = seed_id;
  p.timestep = timestep;
  p.max_a = c->opt.max_a;
  p.ld = c->opt.max_n;
  p.count = 1;
  p.step = nullptr;
  p.capV32 = c->capV32;
  p.slotV32 = c->slotV32;
  cudaError_t e = kp::launch_factor(p, c->stream);
  if (e != cudaSuccess) return kp::cuda_error(c, e, "store_basis launch");
  c->slot_timestep[seed_id] = timestep;
  return KP_OK;
}

kp_status kp_project_targets_multi(kp_ctx* c, int timestep, int nt, const int* seed_ids,
                                   const kp_op* ops, const double* const* r, double* const* x) {
  if (!c) return KP_ERR_ARG;
  int nmax = 0;
  kp_status st = check_ops(c, nt, ops, &nmax);
  if (st != KP_OK) return st;
  if (nt == 0) return KP_OK;
  if (!seed_ids || !r || !x) return kp::set_error(c, KP_ERR_ARG, "seed_ids, r or x is NULL");
  std::vector<SysDesc> h(nt);
  for (int k = 0; k < nt; ++k) {
    const int s = seed_ids[k];
    if (s < 0 || s >= c->opt.max_seeds) return kp::set_error(c, KP_ERR_ARG, "target %d: seed_id %d out of range", k, s);
    if (c->slot_timestep[s] != timestep)
      return kp::set_error(c, KP_ERR_NO_BASIS, "target %d: seed %d holds no basis for timestep %d", k, s, timestep);
    if (!r[k] || !x[k]) return kp::set_error(c, KP_ERR_ARG, "target %d: NULL vector", k);
    h[k] = make_desc(ops[k], r[k], x[k], s);
  }
  int ept = 16, nt_ = 1024;                       // N <= 16384
  if (nmax <= 1024) { ept = 4; nt_ = 256; }
  else if (nmax <= 4096) { ept = 8; nt_ = 512; }
  SysDesc* dd;
  st = upload(c, h, &dd);
  if (st != KP_OK) return st;
  kp::ProjParams p{};
  p.sys = dd;
  p.nt = nt;
  p.timestep = timestep;
  p.slotV = c->slotV;
  p.meta = c->slotMeta;
  p.slotR = c->slotR;
  p.slotRot = c->slotRot;
  p.max_a = c->opt.max_a;
  p.ld = c->opt.max_n;
  p.slotV32 = c->slotV32;
  cudaError_t e = kp::launch_project_fp64(p, ept, nt_, c->stream);
  return e == cudaSuccess ? KP_OK : kp::cuda_error(c, e, "projection launch");
}

kp_status kp_project_targets(kp_ctx* c, int seed_id, int timestep, int nt, const kp_op* ops,
                             const double* const* r, double* const* x) {
  if (!c) return KP_ERR_ARG;
  if (nt < 0) return kp::set_error(c, KP_ERR_ARG, "nt < 0");
  std::vector<int> ids(nt, seed_id);
  return kp_project_targets_multi(c, timestep, nt, ids.data(), ops, r, x);
}

kp_status kp_project_gemm_bf16(kp_ctx* c, int nt, int nv, int K, const void* B, int ldb,
                               const void* V, int ldv, float* C, int ldc) {
  if (!c) return KP_ERR_ARG;
  if (nt < 0 || nv < 1 || nv > 48 || K < 1 || ldb < K || ldv < K || ldc < nv || (ldb % 8) ||
      (ldv % 8) || ((uintptr_t)B % 16) || ((uintptr_t)V % 16) || !C)
    return kp::set_error(c, KP_ERR_ARG, "projection GEMM: bad sizes, strides or alignment");
  if (nt == 0) return KP_OK;
  const int ntiles = (nt + 127) / 128;
  std::vector<kp::ProjTile> tiles(ntiles);
  for (int t = 0; t < ntiles; ++t) {
    tiles[t].row0 = 128 * t;
    tiles[t].vrow0 = 0;
    tiles[t].crow0 = 128 * t;
    tiles[t].count = std::min(128, nt - 128 * t);
    tiles[t].nv = nv;
    tiles[t].ccol0 = 0;
    tiles[t].kc0 = tiles[t].kc1 = 0;
    tiles[t].atomic = 0;
  }
  cudaError_t e = grow(&c->d_tiles, &c->d_tiles_bytes, tiles.size() * sizeof(kp::ProjTile));
  if (e == cudaSuccess && !c->d_err) {
    e = cudaMalloc((void**)&c->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(c->d_err, 0, sizeof(int));
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->d_tiles, tiles.data(), tiles.size() * sizeof(kp::ProjTile),
                        cudaMemcpyHostToDevice, c->stream);
  alignas(64) CUtensorMap mb, mv;
  if (e == cudaSuccess) e = kp::make_bf16_map(&mb, B, nt, K, ldb, 128);
  if (e == cudaSuccess) e = kp::make_bf16_map(&mv, V, nv, K, ldv, 48);
  if (e == cudaSuccess)
    e = kp::launch_proj_gemm_bf16(mb, mv, c->d_tiles, ntiles, K, C, ldc, c->d_err,
                                  std::min(ntiles, c->sms), c->stream);
  return e == cudaSuccess ? KP_OK : kp::cuda_error(c, e, "projection GEMM");
}

kp_status kp_basis_get(kp_ctx* c, int seed_id, int timestep, int* a_out, int* has_next_out,
                       double* V, double* Hbar) {
  if (!c) return KP_ERR_ARG;
  if (seed_id < 0 || seed_id >= c->opt.max_seeds) return kp::set_error(c, KP_ERR_ARG, "seed_id out of range");
  if (c->slot_timestep[seed_id] != timestep)
    return kp::set_error(c, KP_ERR_NO_BASIS, "seed %d holds no basis for timestep %d", seed_id, timestep);
  SlotMeta mt;
  cudaError_t e = cudaMemcpyAsync(&mt, c->slotMeta + seed_id, sizeof(mt), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return kp::cuda_error(c, e, "basis metadata");
  if (a_out) *a_out = mt.a;
  if (has_next_out) *has_next_out = mt.has_next;
  const int a = c->opt.max_a;
  if (V && c->slotV32) {
    e = kp::launch_widen(c->slotV32 + (size_t)seed_id * (a + 1) * c->opt.max_n, c->opt.max_n, V,
                         mt.N, mt.N, mt.a + mt.has_next, c->stream);
    if (e != cudaSuccess) return kp::cuda_error(c, e, "basis copy");
  } else if (V) {
    const int nv = mt.a + mt.has_next;
    e = cudaMemcpy2DAsync(V, (size_t)mt.N * sizeof(double),
                          c->slotV + (size_t)seed_id * (a + 1) * c->opt.max_n,
                          (size_t)c->opt.max_n * sizeof(double), (size_t)mt.N * sizeof(double), nv,
                          cudaMemcpyDeviceToDevice, c->stream);
    if (e != cudaSuccess) return kp::cuda_error(c, e, "basis copy");
  }
  if (Hbar) {
    std::vector<double> tmp((size_t)(a + 1) * a);
    e = cudaMemcpyAsync(tmp.data(), c->slotH + (size_t)seed_id * (a + 1) * a, tmp.size() * sizeof(double),
                        cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return kp::cuda_error(c, e, "Hessenberg copy");
    for (int j = 0; j < mt.a; ++j)
      for (int i = 0; i <= mt.a; ++i) Hbar[i + (size_t)j * (mt.a + 1)] = tmp[i + (size_t)j * (a + 1)];
  }
  if (V) {
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return kp::cuda_error(c, e, "basis copy");
  }
  return KP_OK;
}

}  // extern "C"
