// kp_march.cu -- the time march of Sec. 2.3 with the two phases of Sec. 3 at
// every timestep, replayed from one CUDA graph per parity of n.
//
// The plan owns two copies of every state plane (ping-pong: the solution of
// step n is written into the buffer that held m^{n-2}), the right-hand sides,
// the per-system results and the device-side timestep counter, so that one
// captured graph serves every even and one every odd timestep; the g^2
// schedule is read on the device at the counter's index.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kp.h"
#include "kp_ctx.h"
#include "kp_internal.cuh"

using kp::SysDesc;

namespace {

enum Stat { kSeedIters = 0, kTgtIters, kTgtMax, kNotConv, kMaxRes, kRefFlops, kSeedFlops, kProjFlops, kNStat };

// FP64 flops of GMRES(m) with CGS2 as implemented, per unknown, for k Arnoldi
// steps: start (residual + norms) 14; per cycle of L steps
// sum_j (9 stencil + 8(j+1) Gram-Schmidt + 5 norm/scale) + 2L update + 12 residual.
__device__ __forceinline__ double gmres_flops_per_unknown(int k, int m) {
  double f = 14.0;
  const int full = k / m, rem = k - full * m;
  const double Lm = m;
  f += full * (4.0 * Lm * Lm + 20.0 * Lm + 12.0);
  if (rem > 0) f += 4.0 * rem * rem + 20.0 * rem + 12.0;
  return f;
}

struct StatsParams {
  const kp_info* infoS;
  const int* nS;           // unknowns per seed system
  int ns;
  const kp_info* infoT;
  const int* nT;
  const int* slotT;        // seed slot per target
  int nt;
  const kp::SlotMeta* meta;
  int m_seed, m;
  int project;
  int* step;
  int n0;
  double* stats;           // [steps][kNStat]
};

__global__ void march_stats_kernel(const StatsParams p) {
  __shared__ double red[kNStat][256];
  double v[kNStat];
  for (int k = 0; k < kNStat; ++k) v[k] = 0.0;
  for (int i = threadIdx.x; i < p.ns; i += blockDim.x) {
    const kp_info in = p.infoS[i];
    v[kSeedIters] += in.iters;
    v[kNotConv] += (in.status != 0);
    v[kSeedFlops] += gmres_flops_per_unknown(in.iters, p.m_seed) * p.nS[i];
  }
  for (int i = threadIdx.x; i < p.nt; i += blockDim.x) {
    const kp_info in = p.infoT[i];
    v[kTgtIters] += in.iters;
    v[kTgtMax] = fmax(v[kTgtMax], (double)in.iters);
    v[kNotConv] += (in.status != 0);
    v[kMaxRes] = fmax(v[kMaxRes], in.rel_res);
    v[kRefFlops] += gmres_flops_per_unknown(in.iters, p.m) * p.nT[i];
    if (p.project) {
      const kp::SlotMeta mt = p.meta[p.slotT[i]];
      v[kProjFlops] += (2.0 * (mt.lsq ? mt.a + 1 : mt.a) + 2.0 * mt.a) * p.nT[i];
    }
  }
  for (int k = 0; k < kNStat; ++k) red[k][threadIdx.x] = v[k];
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < kNStat; ++k) {
        const double a = red[k][threadIdx.x], b = red[k][threadIdx.x + s];
        red[k][threadIdx.x] = (k == kTgtMax || k == kMaxRes) ? fmax(a, b) : a + b;
      }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int st = *p.step;
    for (int k = 0; k < kNStat; ++k) p.stats[(size_t)(st - p.n0) * kNStat + k] = red[k][0];
    *p.step = st + 1;
  }
}

template <typename T>
cudaError_t dmalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
}

}  // namespace

struct kp_march_plan {
  kp_ctx* ctx = nullptr;
  kp_march_opts opt{};
  cudaStream_t st = nullptr;
  int ns = 0, nt = 0;
  size_t seed_elems = 0, tgt_elems = 0;
  std::vector<kp_group> groups;
  std::vector<size_t> seed_off, tgt_off;     // element offsets of each group's planes
  // device state
  double* S[2] = {nullptr, nullptr};
  double* Tt[2] = {nullptr, nullptr};
  double* bS = nullptr;
  double* bT = nullptr;
  kp_info* infoS = nullptr;
  kp_info* infoT = nullptr;
  int* nS = nullptr;
  int* nT = nullptr;
  int* slotT = nullptr;
  double* g2 = nullptr;
  int* step = nullptr;
  double* stats = nullptr;
  double* capV = nullptr;
  double* capH = nullptr;
  kp::CapMeta* capMeta = nullptr;
  double* spill = nullptr;
  SysDesc* desc[2] = {nullptr, nullptr};     // per parity: seedRhs, seedSolve, tgtRhs, tgtProj, tgtSolve
  kp::Shape shS, shT;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int launches_per_step = 0;
  int n0_host = 0;           // source of the counter reset (outlives the async copy)
};

namespace {

// Offsets of the descriptor sub-arrays inside desc[parity].
struct DescLayout {
  size_t seedRhs, seedSolve, tgtRhs, tgtProj, tgtSolve, total;
};

DescLayout layout(int ns, int nt) {
  DescLayout L;
  L.seedRhs = 0;
  L.seedSolve = ns;
  L.tgtRhs = 2 * (size_t)ns;
  L.tgtProj = L.tgtRhs + nt;
  L.tgtSolve = L.tgtProj + nt;
  L.total = L.tgtSolve + nt;
  return L;
}

// Enqueue timestep work for parity `par` (state read from buffer par, written
// to buffer 1-par).  ev != null: bracket the kernels with events
// (ev[0..7] = seed start/end, store start/end, proj start/end, refine start/end).
kp_status enqueue_step(kp_march_plan* P, int par, cudaEvent_t* ev, int* launches) {
  kp_ctx* c = P->ctx;
  const DescLayout L = layout(P->ns, P->nt);
  SysDesc* D = P->desc[par];
  double* nxtS = P->S[1 - par];
  double* curT = P->Tt[par];
  double* nxtT = P->Tt[1 - par];
  cudaError_t e = cudaSuccess;
  int nl = 0;
  auto rec = [&](int k) { if (ev && e == cudaSuccess) e = cudaEventRecord(ev[k], P->st); };
  // ---- Phase 1: seeds
  if (P->ns > 0) {
    e = kp::launch_apply(D + L.seedRhs, P->ns, 1, P->st); ++nl;
    if (e == cudaSuccess) e = cudaMemsetAsync(nxtS, 0, P->seed_elems * sizeof(double), P->st);
    rec(0);
    kp::GmresParams g{};
    g.sys = D + L.seedSolve;
    g.nsys = P->ns;
    g.tol = P->opt.tol_seed;
    g.m = P->opt.m_seed;
    g.maxit = P->opt.maxit;
    g.S = P->shS.S;
    g.reorth = c->opt.reorth;
    g.npad = P->shS.ept * P->shS.nt;
    g.spill = (P->shS.S < g.m + 1) ? P->spill : nullptr;
    g.info = P->infoS;
    g.capV = P->capV;
    g.capH = P->capH;
    g.capMeta = P->capMeta;
    g.cap_a = c->opt.max_a;
    g.cap_ld = c->opt.max_n;
    g.step = P->step;
    g.g2_sched = P->g2;
    if (e == cudaSuccess) { e = kp::launch_gmres_fp64(g, P->shS.ept, P->shS.nt, P->shS.smem, P->st); ++nl; }
    rec(1);
    rec(2);
    kp::FactorParams f{};
    f.capV = P->capV;
    f.capH = P->capH;
    f.capMeta = P->capMeta;
    f.sys = 0;
    f.cap_a = c->opt.max_a;
    f.cap_ld = c->opt.max_n;
    f.slotV = c->slotV;
    f.meta = c->slotMeta;
    f.slotR = c->slotR;
    f.slotRot = c->slotRot;
    f.slotH = c->slotH;
    f.seed_id = 0;
    f.timestep = 0;
    f.max_a = c->opt.max_a;
    f.ld = c->opt.max_n;
    f.count = P->ns;
    f.step = P->step;
    if (e == cudaSuccess) { e = kp::launch_factor(f, P->st); ++nl; }
    rec(3);
  }
  // ---- Phase 2: targets
  if (P->nt > 0) {
    if (e == cudaSuccess) { e = kp::launch_apply(D + L.tgtRhs, P->nt, 1, P->st); ++nl; }
    rec(4);
    if (e == cudaSuccess) {
      if (P->opt.mode == KP_MARCH_WARM)
        e = cudaMemcpyAsync(nxtT, curT, P->tgt_elems * sizeof(double), cudaMemcpyDeviceToDevice, P->st);
      else
        e = cudaMemsetAsync(nxtT, 0, P->tgt_elems * sizeof(double), P->st);
    }
    if (P->opt.mode == KP_MARCH_PROJECTED && P->ns > 0 && e == cudaSuccess) {
      kp::ProjParams pp{};
      pp.sys = D + L.tgtProj;
      pp.nt = P->nt;
      pp.timestep = 0;
      pp.slotV = c->slotV;
      pp.meta = c->slotMeta;
      pp.slotR = c->slotR;
      pp.slotRot = c->slotRot;
      pp.max_a = c->opt.max_a;
      pp.ld = c->opt.max_n;
      pp.step = P->step;
      e = kp::launch_project_fp64(pp, P->shT.ept, P->shT.nt, P->st);
      ++nl;
    }
    rec(5);
    rec(6);
    kp::GmresParams g{};
    g.sys = D + L.tgtSolve;
    g.nsys = P->nt;
    g.tol = P->opt.tol;
    g.m = P->opt.m;
    g.maxit = P->opt.maxit;
    g.S = P->shT.S;
    g.reorth = c->opt.reorth;
    g.npad = P->shT.ept * P->shT.nt;
    g.spill = (P->shT.S < g.m + 1) ? P->spill : nullptr;
    g.info = P->infoT;
    g.step = P->step;
    g.g2_sched = P->g2;
    if (e == cudaSuccess) { e = kp::launch_gmres_fp64(g, P->shT.ept, P->shT.nt, P->shT.smem, P->st); ++nl; }
    rec(7);
  }
  StatsParams sp{};
  sp.infoS = P->infoS;
  sp.nS = P->nS;
  sp.ns = P->ns;
  sp.infoT = P->infoT;
  sp.nT = P->nT;
  sp.slotT = P->slotT;
  sp.nt = P->nt;
  sp.meta = c->slotMeta;
  sp.m_seed = P->opt.m_seed;
  sp.m = P->opt.m;
  sp.project = (P->opt.mode == KP_MARCH_PROJECTED && P->ns > 0);
  sp.step = P->step;
  sp.n0 = 0;
  sp.stats = P->stats;
  if (e == cudaSuccess) {
    march_stats_kernel<<<1, 256, 0, P->st>>>(sp);
    e = cudaGetLastError();
    ++nl;
  }
  if (launches) *launches = nl;
  return e == cudaSuccess ? KP_OK : kp::cuda_error(c, e, "march step enqueue");
}

}  // namespace

extern "C" {

kp_status kp_march_destroy(kp_march_plan* P) {
  if (!P) return KP_OK;
  if (P->st) cudaStreamSynchronize(P->st);
  for (auto& g : P->graph)
    if (g) cudaGraphExecDestroy(g);
  for (int k = 0; k < 2; ++k) {
    cudaFree(P->S[k]);
    cudaFree(P->Tt[k]);
    cudaFree(P->desc[k]);
  }
  cudaFree(P->bS); cudaFree(P->bT); cudaFree(P->infoS); cudaFree(P->infoT);
  cudaFree(P->nS); cudaFree(P->nT); cudaFree(P->slotT); cudaFree(P->g2); cudaFree(P->step);
  cudaFree(P->stats); cudaFree(P->capV); cudaFree(P->capH); cudaFree(P->capMeta); cudaFree(P->spill);
  if (P->st) cudaStreamDestroy(P->st);
  delete P;
  return KP_OK;
}

kp_status kp_march_create(kp_ctx* c, int ngroups, const kp_group* groups, const kp_march_opts* opt,
                          kp_march_plan** out) {
  if (!c || !out || !opt || ngroups < 1 || !groups) return c ? kp::set_error(c, KP_ERR_ARG, "bad march arguments") : KP_ERR_ARG;
  *out = nullptr;
  if (c->opt.precision != KP_PREC_FP64)
    return kp::set_error(c, KP_ERR_UNSUPPORTED, "precision mode %d not built in the march", c->opt.precision);
  const kp_march_opts& o = *opt;
  if (o.T < 1 || !o.g2 || o.mode < 0 || o.mode > 2 || o.m_seed < 1 || o.m_seed > kp::kMaxM ||
      o.m < 1 || o.m > kp::kMaxM || o.maxit < 0 || !(o.tol >= 0) || !(o.tol_seed >= 0))
    return kp::set_error(c, KP_ERR_ARG, "bad march options");
  kp_march_plan* P = new kp_march_plan();
  P->ctx = c;
  P->opt = o;
  P->groups.assign(groups, groups + ngroups);
  int nmaxS = 0, nmaxT = 0;
  for (int gi = 0; gi < ngroups; ++gi) {
    const kp_group& g = groups[gi];
    const int N = g.H * g.W;
    if (g.H < 1 || g.W < 1 || N > c->opt.max_n || g.nseed < 0 || g.ntgt < 0 ||
        (g.nseed && !g.m_seed) || (g.ntgt && !g.m_tgt) || (g.ntgt && !g.tgt_seed)) {
      kp_march_destroy(P);
      return kp::set_error(c, KP_ERR_ARG, "group %d: bad sizes or pointers", gi);
    }
    for (int t = 0; t < g.ntgt; ++t)
      if (g.tgt_seed[t] < 0 || g.tgt_seed[t] >= g.nseed) {
        if (o.mode == KP_MARCH_PROJECTED) {
          kp_march_destroy(P);
          return kp::set_error(c, KP_ERR_ARG, "group %d target %d: seed index out of range", gi, t);
        }
      }
    P->seed_off.push_back(P->seed_elems);
    P->tgt_off.push_back(P->tgt_elems);
    P->seed_elems += (size_t)g.nseed * N;
    P->tgt_elems += (size_t)g.ntgt * N;
    P->ns += g.nseed;
    P->nt += g.ntgt;
    if (g.nseed) nmaxS = std::max(nmaxS, N);
    if (g.ntgt) nmaxT = std::max(nmaxT, N);
  }
  if (P->ns > c->opt.max_seeds) {
    kp_march_destroy(P);
    return kp::set_error(c, KP_ERR_ARG, "%d seeds exceed max_seeds=%d", P->ns, c->opt.max_seeds);
  }
  kp_status s = KP_OK;
  if (P->ns) s = kp::gmres_shape(c, nmaxS, o.m_seed, &P->shS);
  if (s == KP_OK && P->nt) s = kp::gmres_shape(c, nmaxT, o.m, &P->shT);
  if (s != KP_OK) { kp_march_destroy(P); return s; }
  cudaError_t e = cudaStreamCreateWithFlags(&P->st, cudaStreamNonBlocking);
  const int ns = P->ns, nt = P->nt;
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = dmalloc(&P->S[k], P->seed_elems);
    if (e == cudaSuccess) e = dmalloc(&P->Tt[k], P->tgt_elems);
  }
  if (e == cudaSuccess) e = dmalloc(&P->bS, P->seed_elems);
  if (e == cudaSuccess) e = dmalloc(&P->bT, P->tgt_elems);
  if (e == cudaSuccess) e = dmalloc(&P->infoS, ns);
  if (e == cudaSuccess) e = dmalloc(&P->infoT, nt);
  if (e == cudaSuccess) e = dmalloc(&P->nS, ns);
  if (e == cudaSuccess) e = dmalloc(&P->nT, nt);
  if (e == cudaSuccess) e = dmalloc(&P->slotT, nt);
  if (e == cudaSuccess) e = dmalloc(&P->g2, o.T);
  if (e == cudaSuccess) e = dmalloc(&P->step, 1);
  if (e == cudaSuccess) e = dmalloc(&P->stats, (size_t)o.T * kNStat);
  if (e == cudaSuccess && ns) {
    e = dmalloc(&P->capV, (size_t)ns * (c->opt.max_a + 1) * c->opt.max_n);
    if (e == cudaSuccess) e = dmalloc(&P->capH, (size_t)ns * (c->opt.max_a + 1) * c->opt.max_a);
    if (e == cudaSuccess) e = dmalloc(&P->capMeta, ns);
  }
  size_t spill = 0;
  if (ns && P->shS.S < o.m_seed + 1)
    spill = std::max(spill, (size_t)ns * (o.m_seed + 1 - P->shS.S) * P->shS.ept * P->shS.nt);
  if (nt && P->shT.S < o.m + 1)
    spill = std::max(spill, (size_t)nt * (o.m + 1 - P->shT.S) * P->shT.ept * P->shT.nt);
  if (e == cudaSuccess && spill) e = dmalloc(&P->spill, spill);
  const DescLayout L = layout(ns, nt);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = dmalloc(&P->desc[k], L.total);
  if (e != cudaSuccess) {
    kp_status r = kp::cuda_error(c, e, "march allocation");
    kp_march_destroy(P);
    return r;
  }
  // host-side tables
  const double dt = 1.0 / o.T;
  std::vector<int> hnS(std::max(ns, 1)), hnT(std::max(nt, 1)), hslot(std::max(nt, 1));
  std::vector<SysDesc> hd[2];
  for (int par = 0; par < 2; ++par) {
    hd[par].resize(L.total);
    double* cS = P->S[par];
    double* xS = P->S[1 - par];
    double* cT = P->Tt[par];
    double* xT = P->Tt[1 - par];
    int si = 0, ti = 0, seed_base = 0;
    for (int gi = 0; gi < ngroups; ++gi) {
      const kp_group& g = groups[gi];
      const int N = g.H * g.W;
      for (int k = 0; k < g.nseed; ++k, ++si) {
        const size_t off = P->seed_off[gi] + (size_t)k * N;
        SysDesc d{};
        d.H = g.H; d.W = g.W; d.dt = dt; d.g2 = 0.0; d.h = 1.0 / g.H;
        d.mt = cS + off; d.fx = d.fy = nullptr;
        d.b = cS + off; d.x = P->bS + off;            // rhs: b <- m^{n-1}/dt
        hd[par][L.seedRhs + si] = d;
        d.b = P->bS + off; d.x = xS + off;            // solve into the other buffer
        hd[par][L.seedSolve + si] = d;
        hnS[si] = N;
      }
      for (int k = 0; k < g.ntgt; ++k, ++ti) {
        const size_t off = P->tgt_off[gi] + (size_t)k * N;
        SysDesc d{};
        d.H = g.H; d.W = g.W; d.dt = dt; d.g2 = 0.0; d.h = 1.0 / g.H;
        d.mt = cT + off; d.fx = d.fy = nullptr;
        d.b = cT + off; d.x = P->bT + off;
        hd[par][L.tgtRhs + ti] = d;
        d.b = P->bT + off; d.x = xT + off;
        const int sd = (g.tgt_seed[k] >= 0 && g.tgt_seed[k] < g.nseed) ? g.tgt_seed[k] : 0;
        d.slot = seed_base + sd;
        hd[par][L.tgtProj + ti] = d;
        d.slot = 0;
        hd[par][L.tgtSolve + ti] = d;
        hnT[ti] = N;
        hslot[ti] = seed_base + sd;
      }
      seed_base += g.nseed;
    }
  }
  for (int k = 0; k < 2 && e == cudaSuccess; ++k)
    e = cudaMemcpy(P->desc[k], hd[k].data(), L.total * sizeof(SysDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(P->nS, hnS.data(), ns * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(P->nT, hnT.data(), nt * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(P->slotT, hslot.data(), nt * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(P->g2, o.g2, o.T * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    kp_status r = kp::cuda_error(c, e, "march tables");
    kp_march_destroy(P);
    return r;
  }
  // graphs: one per parity
  if (o.use_graph) {
    for (int par = 0; par < 2; ++par) {
      cudaGraph_t gr = nullptr;
      e = cudaStreamBeginCapture(P->st, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) break;
      kp_status r = enqueue_step(P, par, nullptr, &P->launches_per_step);
      cudaError_t e2 = cudaStreamEndCapture(P->st, &gr);
      if (r != KP_OK) { if (gr) cudaGraphDestroy(gr); kp_march_destroy(P); return r; }
      e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&P->graph[par], gr, 0);
      if (gr) cudaGraphDestroy(gr);
      if (e != cudaSuccess) break;
    }
    if (e != cudaSuccess) {
      kp_status r = kp::cuda_error(c, e, "march graph capture");
      kp_march_destroy(P);
      return r;
    }
  }
  *out = P;
  return KP_OK;
}

kp_status kp_march_run(kp_march_plan* P, int n0, int steps, kp_step_stats* stats,
                       kp_march_timing* timing) {
  if (!P) return KP_ERR_ARG;
  kp_ctx* c = P->ctx;
  if (n0 < 0 || steps < 0 || n0 + steps > P->opt.T)
    return kp::set_error(c, KP_ERR_ARG, "timesteps %d..%d outside 1..%d", n0 + 1, n0 + steps, P->opt.T);
  if (steps == 0) return KP_OK;
  cudaError_t e = cudaSuccess;
  // order after the caller's stream, then copy the caller's states in
  cudaEvent_t join = nullptr;
  e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(join, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(P->st, join, 0);
  for (size_t gi = 0; gi < P->groups.size() && e == cudaSuccess; ++gi) {
    const kp_group& g = P->groups[gi];
    const size_t N = (size_t)g.H * g.W;
    if (g.nseed) e = cudaMemcpyAsync(P->S[0] + P->seed_off[gi], g.m_seed, g.nseed * N * sizeof(double), cudaMemcpyDeviceToDevice, P->st);
    if (e == cudaSuccess && g.ntgt) e = cudaMemcpyAsync(P->Tt[0] + P->tgt_off[gi], g.m_tgt, g.ntgt * N * sizeof(double), cudaMemcpyDeviceToDevice, P->st);
  }
  P->n0_host = n0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(P->step, &P->n0_host, sizeof(int), cudaMemcpyHostToDevice, P->st);
  std::vector<cudaEvent_t> ev;
  int launches = 0;
  if (e == cudaSuccess && timing) {
    ev.resize((size_t)steps * 8, nullptr);
    for (auto& x : ev)
      if (e == cudaSuccess) e = cudaEventCreate(&x);
  }
  kp_status r = KP_OK;
  for (int k = 0; k < steps && e == cudaSuccess && r == KP_OK; ++k) {
    const int par = k & 1;
    if (timing) {
      int nl = 0;
      r = enqueue_step(P, par, ev.data() + (size_t)k * 8, &nl);
      launches += nl;
    } else if (P->graph[par]) {
      e = cudaGraphLaunch(P->graph[par], P->st);
      launches += P->launches_per_step;
    } else {
      int nl = 0;
      r = enqueue_step(P, par, nullptr, &nl);
      launches += nl;
    }
  }
  // states back to the caller's buffers
  const int fin = steps & 1;
  for (size_t gi = 0; gi < P->groups.size() && e == cudaSuccess && r == KP_OK; ++gi) {
    const kp_group& g = P->groups[gi];
    const size_t N = (size_t)g.H * g.W;
    if (g.nseed) e = cudaMemcpyAsync(g.m_seed, P->S[fin] + P->seed_off[gi], g.nseed * N * sizeof(double), cudaMemcpyDeviceToDevice, P->st);
    if (e == cudaSuccess && g.ntgt) e = cudaMemcpyAsync(g.m_tgt, P->Tt[fin] + P->tgt_off[gi], g.ntgt * N * sizeof(double), cudaMemcpyDeviceToDevice, P->st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(join, P->st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, join, 0);
  if (e == cudaSuccess && (stats || timing)) e = cudaStreamSynchronize(P->st);
  if (e == cudaSuccess && stats) {
    std::vector<double> h((size_t)steps * kNStat);
    e = cudaMemcpy(h.data(), P->stats + (size_t)n0 * kNStat, h.size() * sizeof(double), cudaMemcpyDeviceToHost);
    for (int k = 0; k < steps && e == cudaSuccess; ++k) {
      const double* v = h.data() + (size_t)k * kNStat;
      stats[k].seed_iters = v[kSeedIters];
      stats[k].tgt_iters = v[kTgtIters];
      stats[k].tgt_iters_max = v[kTgtMax];
      stats[k].not_converged = v[kNotConv];
      stats[k].max_rel_res = v[kMaxRes];
      stats[k].refine_flops = v[kRefFlops];
      stats[k].seed_flops = v[kSeedFlops];
      stats[k].proj_flops = v[kProjFlops];
    }
  }
  if (e == cudaSuccess && timing) {
    std::memset(timing, 0, sizeof(*timing));
    for (int k = 0; k < steps && e == cudaSuccess; ++k) {
      cudaEvent_t* x = ev.data() + (size_t)k * 8;
      float a = 0, b = 0, cc = 0, d = 0, s = 0;
      if (P->ns) {
        e = cudaEventElapsedTime(&a, x[0], x[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&b, x[2], x[3]);
      }
      if (e == cudaSuccess && P->nt) {
        e = cudaEventElapsedTime(&cc, x[4], x[5]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&d, x[6], x[7]);
      }
      if (e == cudaSuccess && P->ns && P->nt) e = cudaEventElapsedTime(&s, x[0], x[7]);
      timing->seed_ms += a;
      timing->store_ms += b;
      timing->proj_ms += cc;
      timing->refine_ms += d;
      timing->step_ms += s;
    }
  }
  if (timing) timing->launches = launches;
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  if (join) cudaEventDestroy(join);
  if (r != KP_OK) return r;
  return e == cudaSuccess ? KP_OK : kp::cuda_error(c, e, "march run");
}

}  // extern "C"
