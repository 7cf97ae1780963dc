// kp_march.cu -- the time march of Sec. 2.3 with the two phases of Sec. 3 at
// every timestep, replayed from one CUDA graph per parity of n.
//
// Per timestep n the graph holds two solver launches on parallel branches:
//   targets of step n: b = m^{n-1}/dt formed on the fly, initial guess by
//     projection onto the seed basis of step n (or 0, or m^{n-1}), GMRES(m);
//   seeds of step n+1: GMRES(m_seed) from 0 with the first-cycle basis
//     written straight into the seed slots of parity n+1 and H_a factored.
// Seeds never depend on targets, so running them one step ahead lets their
// (latency-bound, few-block) solves fill the SMs the target wave leaves idle.
// A one-thread kernel then advances the device-side timestep counter, from
// which both launches read g^2 and their slot parity; two copies of every
// state plane alternate by parity, so one graph serves all even and one all
// odd timesteps.
//
// FP64 plans march in windows of K timesteps instead: one graph replay runs
// the seeds of window w+1 (each seed block marches its system through the K
// steps, writing slot set t mod 2K) and, started programmatically beside
// them, one persistent target launch over the K x (targets) items of window w.  Target blocks claim items from a
// counter in timestep-major order, so the launch has no per-timestep wave
// tail; an item waits (bounded) only for its own system's previous timestep,
// which an earlier claim -- a running block -- is solving.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kp.h"
#include "kp_ctx.h"
#include "kp_internal.cuh"

using kp::SysDesc;

namespace {

template <typename T>
cudaError_t dmalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
}

}  // namespace

struct kp_march_plan {
  kp_ctx* ctx = nullptr;
  kp_march_opts opt{};
  cudaStream_t st = nullptr;         // main branch (targets) and graph launches
  cudaStream_t st2 = nullptr;        // seed branch inside the captured graph
  cudaEvent_t fork = nullptr, join = nullptr;
  int ns = 0, nt = 0;
  size_t seed_elems = 0, tgt_elems = 0;
  std::vector<kp_group> groups;
  std::vector<size_t> seed_off, tgt_off;     // element offsets of each group's planes
  // device state
  double* S[2] = {nullptr, nullptr};        // seed states, m_s^k in S[k & 1]
  double* Tt[2] = {nullptr, nullptr};       // target states, m_t^k in Tt[k & 1]
  double* g2 = nullptr;
  int* step = nullptr;                      // [0] current target timestep, [1] end of run
  kp::StepAcc* acc = nullptr;               // [T]
  double* spill = nullptr;
  float* spill32 = nullptr;
  bool mixed = false;
  // targets are stored sorted by seed so that a seed's targets form whole
  // tensor-core tiles: internal plane q of group g holds user plane perm[q]
  int* perm = nullptr;                       // device, group-local indices
  std::vector<int> tgt_base;                 // first internal target of each group
  // tensor-core projection (mixed precision)
  __nv_bfloat16* Bb = nullptr;               // [nt][vb_ld] BF16 right-hand sides
  float* Cp = nullptr;                       // [nt][kVbRows] projections c = V^T b
  kp::ProjTile* tiles[2] = {nullptr, nullptr};
  std::vector<int> tile_off, tile_cnt;       // per group, within each parity's list
  std::vector<CUtensorMap> mapB, mapV;       // per group
  int* err = nullptr;
  int gemm_grid = 0;
  // exact Galerkin in mixed precision: per-timestep Gram matrices with the
  // target-dependent part on the tensor cores (kp_gram.cu)
  int gram_A = 0, p_ld = 0, q_ld = 0;
  __nv_bfloat16* Pb = nullptr;               // [2 ns A^2][p_ld] product rows of the seed bases
  float* G0 = nullptr;                       // [2 ns][A^2]
  __nv_bfloat16* Qb = nullptr;               // [nt][q_ld] coefficient rows of the targets
  float* Cg = nullptr;                       // [nt][A^2] = Q P^T
  kp::ProjTile* gtiles[2] = {nullptr, nullptr};
  std::vector<int> gtile_off, gtile_cnt;     // per group
  std::vector<CUtensorMap> mapQ, mapP;       // per group
  SysDesc* desc[2] = {nullptr, nullptr};     // per parity p: seeds (step n+1), targets (step n)
  kp::Shape shS, shT;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int launches_per_step = 0;
  int host_step[3] = {0, 0, 0};              // source of the counter reset (outlives the copy)
  // windows of K timesteps (FP64): K = 1 is the per-timestep scheme above
  int K = 1;
  int* queue = nullptr;                      // [2] item counters of the target launches
  int* done = nullptr;                       // [nt] steps completed in this run
  // target classes: in window mode, grids of <= 1024 points and larger ones
  // get their own solver shape and persistent launch (targets of a class are
  // contiguous in the descriptor arrays); otherwise one class = all targets
  struct TClass {
    kp::Shape sh;
    int first = 0, count = 0, grid = 0;
    size_t spill_off = 0;                    // in the target part of the workspace
  };
  int ncls = 1;
  TClass cls[2];
  size_t score_stride = 0;                   // elements per timestep of the score output
  // seed cycling: predecessor of each plan seed (device), the lagged field of
  // each slot's seed solve, and the served slots the targets read
  bool cycling = false;
  int* cyc_prev = nullptr;                   // [ns]
  double* slotM = nullptr;                   // [max_seeds][max_n]
  double* cycV = nullptr;                    // [max_seeds][max_a + 1][max_n]
  double* cycR = nullptr;                    // [max_seeds][(max_a + 1) * max_a]
  kp::SlotMeta* cycMeta = nullptr;           // [max_seeds]
  float* cycS = nullptr;                     // [K * ns][max_a][max_n] FP32 workspace
  // learned guess: per parity, device tables of the targets' m^{n-1} and their
  // seeds' m_seed^n, internal order
  kp_cnn* cnn = nullptr;
  const double** lg_prev[2] = {nullptr, nullptr};
  const double** lg_seed[2] = {nullptr, nullptr};
  float* gdelta = nullptr;                   // [nt][H W] network output of the step's targets
  double* grho = nullptr;                    // [nt] their step-residual rms
};

namespace {

kp::GmresParams solver_params(kp_march_plan* P, bool seeds, int par, int offset, int ci = 0) {
  kp_ctx* c = P->ctx;
  kp::GmresParams g{};
  const kp_march_plan::TClass& tc = P->cls[ci];
  const kp::Shape& sh = seeds ? P->shS : tc.sh;
  const int first = seeds ? 0 : P->ns + tc.first;
  g.sys = P->desc[par] + first;
  g.nsys = seeds ? P->ns : tc.count;
  g.tol = seeds ? P->opt.tol_seed : P->opt.tol;
  g.m = seeds ? P->opt.m_seed : P->opt.m;
  g.maxit = seeds && P->opt.maxit_seed > 0 ? P->opt.maxit_seed : P->opt.maxit;
  g.S = sh.S;
  g.reorth = c->opt.reorth;
  g.inner_eta = kp::inner_eta(c->opt);
  g.npad = sh.ept * sh.nt;
  size_t spS = 0;
  if (P->ns && P->shS.S < P->opt.m_seed + 1)
    spS = (size_t)P->ns * (P->shS.cs ? P->shS.cs : 1) * (P->opt.m_seed + 1 - P->shS.S) * P->shS.ept *
          P->shS.nt;
  if (P->mixed)
    g.spill32 = (sh.S < g.m + 1) ? P->spill32 + (seeds ? 0 : spS + tc.spill_off) : nullptr;
  else
    g.spill = (sh.S < g.m + 1) ? P->spill + (seeds ? 0 : spS + tc.spill_off) : nullptr;
  g.slotV32 = c->slotV32;
  g.info = nullptr;
  g.step = P->step;
  g.g2_sched = P->g2;
  g.step_offset = offset;
  g.step_end = P->step + 1;
  g.b_scale = (double)P->opt.T;               // b = m^{n-1} / dt with dt = 1/T
  g.slotV = c->slotV;
  g.slotMeta = c->slotMeta;
  g.slotR = c->slotR;
  g.slotRot = c->slotRot;
  g.slot_ld = c->opt.max_n;
  g.max_a = c->opt.max_a;
  g.slot_parity_stride = P->ns;
  g.acc = P->acc;
  g.err = P->err;
  g.picard = P->opt.picard;
  g.bicg = P->opt.seed_solver == KP_SEED_BICGSTAB;
  g.dense_slots = !seeds && (g.bicg || P->cycling);
  if (seeds) g.capM = P->slotM;
  if (!seeds && P->cycling) {                // targets read the served slots
    g.slotV = P->cycV;
    g.slotMeta = P->cycMeta;
    g.slotR = P->cycR;
  }
  if (P->K > 1) {
    // window: descriptors and slot sets chosen per timestep on the device
    g.win = P->K;
    g.slot_sets = 2 * P->K;
    g.sys_par[0] = P->desc[0] + first;
    g.sys_par[1] = P->desc[1] + first;
    g.sys_shift = seeds ? 1 : 0;
    g.step_offset = seeds ? offset : 0;
    if (!seeds) {
      g.queue = P->queue + ci;
      g.done = P->done + tc.first;
      g.run_start = P->step + 2;
      if (P->opt.wait_probe) {               // testing aid: every wait runs out, quickly
        g.wait_bias = 1;
        g.wait_limit = 1 << 14;
      }
      g.grid = tc.grid;
    }
  }
  if (seeds) {
    g.x0_mode = kp::X0_ZERO;
    if (P->mixed) {
      g.capV32 = c->slotV32;                 // capture straight into the seed slots
      g.capVb = c->slotVb;                   // and its BF16 copy for the tensor cores
      g.capVb_ld = c->vb_ld;
    } else {
      g.capV = c->slotV;
    }
    g.capH = c->slotH;
    g.cap_a = c->opt.max_a;
    g.cap_ld = c->opt.max_n;
    g.fixed_a = c->opt.fixed_a;
    g.factor = 1;
    g.acc_kind = 0;
  } else {
    g.score_stride = P->score_stride;
    g.x0_mode = P->opt.mode == KP_MARCH_PROJECTED ? (P->ns ? kp::X0_PROJECT : kp::X0_ZERO)
              : P->opt.mode == KP_MARCH_GALERKIN ? (P->ns ? kp::X0_GALERKIN : kp::X0_ZERO)
              : P->opt.mode == KP_MARCH_LEARNED ? kp::X0_GUESS_PROJECT
              : P->opt.mode == KP_MARCH_LEARNED_ONLY ? kp::X0_READ
              : P->opt.mode == KP_MARCH_WARM ? kp::X0_WARM : kp::X0_ZERO;
    g.acc_kind = 1;
    if (P->Cp) {
      g.cproj = P->Cp;                       // c = V^T b from the tensor-core GEMM
      g.cproj_ld = kp::kVbRows;
      g.bnext = P->Bb;                       // BF16 b of the next timestep
      g.bnext_ld = c->vb_ld;
    }
    if (P->G0) {
      g.gram0 = P->G0;                       // Galerkin: G = G0 (seed basis) + C (target)
      g.gram = P->Cg;
      g.gram_a = P->gram_A;
    }
    if (P->gdelta) {                         // learned guess: x_init = m + (rho / T) net
      g.gdelta = P->gdelta;
      g.gdelta_ld = P->groups[0].H * P->groups[0].W;
      g.grho = P->grho;
      g.gdiv = (double)P->opt.T;
    }
  }
  return g;
}

cudaError_t launch_solver(kp_march_plan* P, const kp::GmresParams& g, const kp::Shape& sh,
                          cudaStream_t st) {
  return kp::launch_solver(g, sh, P->mixed, st);
}

// Seed cycling for the timesteps of the seed launch with the same offset
// (window: K of them; per-timestep scheme: one): the served slots.
cudaError_t launch_cycle(kp_march_plan* P, int offset, cudaStream_t st) {
  if (!P->cycling) return cudaSuccess;
  kp_ctx* c = P->ctx;
  kp::CycleParams q{};
  q.sys = P->desc[0];
  q.prev = P->cyc_prev;
  q.ns = P->ns;
  q.slotV = c->slotV;
  q.slotMeta = c->slotMeta;
  q.slotR = c->slotR;
  q.slotM = P->slotM;
  q.outV = P->cycV;
  q.outMeta = P->cycMeta;
  q.outR = P->cycR;
  q.max_a = c->opt.max_a;
  q.ld = c->opt.max_n;
  q.step = P->step;
  q.step_offset = offset;
  q.win = P->K;
  q.step_end = P->step + 1;
  q.g2_sched = P->g2;
  q.b_scale = (double)P->opt.T;                 // as the solvers' b_scale
  q.slot_sets = P->K > 1 ? 2 * P->K : 0;
  q.scratch = P->cycS;
  int nmax = 0;
  for (const kp_group& g : P->groups)
    if (g.nseed) nmax = std::max(nmax, g.H * g.W);
  return kp::launch_cycle(q, nmax, P->K * P->ns, st);
}

// The learned guess of the targets of step n (parity par): pack, network and
// x_init = m^{n-1} + s_n * net into the solver's output planes, in passes of
// the network's inference batch.
cudaError_t enqueue_guess(kp_march_plan* P, int par, int* nl) {
  const int B = kp::cnn_inference_batch(P->cnn);
  cudaError_t e = cudaSuccess;
  for (int c0 = 0; c0 < P->nt && e == cudaSuccess; c0 += B) {
    const size_t plane = (size_t)P->groups[0].H * P->groups[0].W;
    e = kp::cnn_enqueue_guess(P->cnn, std::min(B, P->nt - c0), P->lg_prev[par] + c0, P->lg_seed[par] + c0,
                              P->gdelta + (size_t)c0 * plane, P->grho + c0, P->step, 0, P->g2, P->opt.T, P->st);
    *nl += 2 + 4;                            // residual rms, pack, four layers (x_init in the solver)
  }
  return e;
}

// Exact Galerkin in mixed precision, targets of step n (parity par): the
// product rows and G0 of the step's seed bases, the targets' coefficient rows,
// and C = Q P^T per group on the tensor cores.
cudaError_t enqueue_gram(kp_march_plan* P, int par, int* nl) {
  kp_ctx* c = P->ctx;
  kp::GramParams gp{};
  gp.seeds = P->desc[par];
  gp.targets = P->desc[par] + P->ns;
  gp.ns = P->ns;
  gp.nt = P->nt;
  gp.A = P->gram_A;
  gp.max_a = c->opt.max_a;
  gp.slot_ld = c->opt.max_n;
  for (const kp_group& g : P->groups) gp.max_n = std::max(gp.max_n, g.H * g.W);
  gp.step = P->step;
  gp.g2_sched = P->g2;
  gp.b_scale = (double)P->opt.T;
  gp.slotMeta = c->slotMeta;
  gp.slotV32 = c->slotV32;
  gp.Pb = P->Pb;
  gp.p_ld = P->p_ld;
  gp.G0 = P->G0;
  gp.Qb = P->Qb;
  gp.q_ld = P->q_ld;
  cudaError_t e = kp::launch_gram_products(gp, P->st);
  if (e == cudaSuccess) e = kp::launch_gram_coeff(gp, P->st);
  *nl += 2;
  for (size_t gi = 0; gi < P->groups.size() && e == cudaSuccess; ++gi) {
    if (!P->gtile_cnt[gi]) continue;
    e = kp::launch_proj_gemm_bf16(P->mapQ[gi], P->mapP[gi], P->gtiles[par] + P->gtile_off[gi], P->gtile_cnt[gi],
                                  2 * P->groups[gi].H * P->groups[gi].W, P->Cg, P->gram_A * P->gram_A, P->err,
                                  std::min(P->gtile_cnt[gi], P->gemm_grid), P->st);
    ++*nl;
  }
  return e;
}

// Target step n and seed step n+1 for parity p = n & 1.  With ev (timing
// mode) the launches run one after the other between events ev[0..1]
// (seeds), ev[4..5] (learned guess) and ev[2..3] (targets); otherwise seeds
// and targets run on two branches.
kp_status enqueue_step(kp_march_plan* P, int par, cudaEvent_t* ev, int* launches) {
  cudaError_t e = cudaSuccess;
  int nl = 0;
  const bool branch = (ev == nullptr) && P->ns > 0 && P->nt > 0;
  cudaStream_t sst = branch ? P->st2 : P->st;
  if (branch) {
    e = cudaEventRecord(P->fork, P->st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->st2, P->fork, 0);
  }
  if (P->ns > 0 && e == cudaSuccess) {
    if (ev) e = cudaEventRecord(ev[0], sst);
    kp::GmresParams g = solver_params(P, true, par, 1);
    if (e == cudaSuccess) e = launch_solver(P, g, P->shS, sst);
    ++nl;
    if (P->cycling && e == cudaSuccess) { e = launch_cycle(P, 1, sst); ++nl; }
    if (ev && e == cudaSuccess) e = cudaEventRecord(ev[1], sst);
  }
  if (P->nt > 0 && P->cnn && e == cudaSuccess) {
    if (ev) e = cudaEventRecord(ev[4], P->st);
    if (e == cudaSuccess) e = enqueue_guess(P, par, &nl);
    if (ev && e == cudaSuccess) e = cudaEventRecord(ev[5], P->st);
  }
  if (P->nt > 0 && e == cudaSuccess) {
    if (ev) e = cudaEventRecord(ev[2], P->st);
    if (P->Cp) {
      for (size_t gi = 0; gi < P->groups.size() && e == cudaSuccess; ++gi) {
        if (!P->tile_cnt[gi]) continue;
        e = kp::launch_proj_gemm_bf16(P->mapB[gi], P->mapV[gi], P->tiles[par] + P->tile_off[gi],
                                      P->tile_cnt[gi], P->groups[gi].H * P->groups[gi].W, P->Cp,
                                      kp::kVbRows, P->err, std::min(P->tile_cnt[gi], P->gemm_grid),
                                      P->st);
        ++nl;
      }
    }
    if (P->G0 && e == cudaSuccess) e = enqueue_gram(P, par, &nl);
    kp::GmresParams g = solver_params(P, false, par, 0);
    if (e == cudaSuccess) e = launch_solver(P, g, P->cls[0].sh, P->st);
    ++nl;
    if (ev && e == cudaSuccess) e = cudaEventRecord(ev[3], P->st);
  }
  if (branch && e == cudaSuccess) {
    e = cudaEventRecord(P->join, P->st2);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(P->st, P->join, 0);
  }
  if (e == cudaSuccess) { e = kp::launch_advance(P->step, P->st); ++nl; }
  if (launches) *launches = nl;
  return e == cudaSuccess ? KP_OK : kp::cuda_error(P->ctx, e, "march step enqueue");
}

// Window of K timesteps from the device counter t0, on one stream: the seeds
// of t0+K..t0+2K-1, then the targets of t0..t0+K-1 as a programmatic
// dependent launch (the seed blocks signal at entry, so the persistent target
// blocks fill every slot the few seed blocks leave and take theirs when the
// seed chains end; targets never read this window's seeds), then t0 += K and
// the item counter reset.  With ev (timing mode) the launches are plain and
// bracketed by ev[0..1] (seeds) and ev[2..3] (targets).
kp_status enqueue_window(kp_march_plan* P, cudaEvent_t* ev, int* launches) {
  cudaError_t e = cudaSuccess;
  int nl = 0;
  const bool pdl = (ev == nullptr) && P->ns > 0 && P->nt > 0;
  if (P->ns > 0) {
    if (ev) e = cudaEventRecord(ev[0], P->st);
    kp::GmresParams g = solver_params(P, true, 0, P->K);
    g.pdl = pdl ? 1 : 0;                     // signal at entry
    if (e == cudaSuccess) e = launch_solver(P, g, P->shS, P->st);
    ++nl;
    // seed cycling of the next window: timed with the seeds; otherwise after
    // the target launch, which keeps its programmatic start on the seeds
    if (ev && P->cycling && e == cudaSuccess) { e = launch_cycle(P, P->K, P->st); ++nl; }
    if (ev && e == cudaSuccess) e = cudaEventRecord(ev[1], P->st);
  }
  if (P->nt > 0 && e == cudaSuccess) {
    if (ev) e = cudaEventRecord(ev[2], P->st);
    // class launches chained the same way: each signals at entry so the next
    // one fills the SMs it leaves, and waits at exit for its predecessor
    for (int ci = 0; ci < P->ncls && e == cudaSuccess; ++ci) {
      kp::GmresParams g = solver_params(P, false, 0, 0, ci);
      if (ev == nullptr) g.pdl = ((P->ns > 0 || ci > 0) ? 2 : 0) | (ci + 1 < P->ncls ? 1 : 0);
      e = launch_solver(P, g, P->cls[ci].sh, P->st);
      ++nl;
    }
    if (ev && e == cudaSuccess) e = cudaEventRecord(ev[3], P->st);
  }
  if (!ev && P->ns > 0 && P->cycling && e == cudaSuccess) { e = launch_cycle(P, P->K, P->st); ++nl; }
  if (e == cudaSuccess) { e = kp::launch_advance(P->step, P->st, P->K, P->queue, P->ncls); ++nl; }
  if (launches) *launches = nl;
  return e == cudaSuccess ? KP_OK : kp::cuda_error(P->ctx, e, "march window enqueue");
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
  cudaFree(P->g2);
  cudaFree(P->step);
  cudaFree(P->acc);
  cudaFree(P->spill);
  cudaFree(P->spill32);
  cudaFree(P->cyc_prev);
  cudaFree(P->slotM);
  cudaFree(P->cycV);
  cudaFree(P->cycR);
  cudaFree(P->cycMeta);
  cudaFree(P->cycS);
  cudaFree(P->perm);
  for (int k = 0; k < 2; ++k) {
    cudaFree(P->lg_prev[k]);
    cudaFree(P->lg_seed[k]);
  }
  cudaFree(P->gdelta);
  cudaFree(P->grho);
  cudaFree(P->Bb);
  cudaFree(P->Cp);
  cudaFree(P->tiles[0]);
  cudaFree(P->tiles[1]);
  cudaFree(P->Pb);
  cudaFree(P->G0);
  cudaFree(P->Qb);
  cudaFree(P->Cg);
  cudaFree(P->gtiles[0]);
  cudaFree(P->gtiles[1]);
  cudaFree(P->err);
  cudaFree(P->queue);
  cudaFree(P->done);
  if (P->fork) cudaEventDestroy(P->fork);
  if (P->join) cudaEventDestroy(P->join);
  if (P->st2) cudaStreamDestroy(P->st2);
  if (P->st) cudaStreamDestroy(P->st);
  delete P;
  return KP_OK;
}

kp_status kp_march_create(kp_ctx* c, int ngroups, const kp_group* groups, const kp_march_opts* opt,
                          kp_march_plan** out) {
  if (!c) return KP_ERR_ARG;
  if (!out || !opt || ngroups < 1 || !groups) return kp::set_error(c, KP_ERR_ARG, "bad march arguments");
  *out = nullptr;
  const kp_march_opts& o = *opt;
  if (o.T < 1 || !o.g2 || o.mode < 0 || o.mode > 5 || o.m_seed < 1 || o.m_seed > kp::kMaxM ||
      (o.score != nullptr) != (o.embed != nullptr) || o.picard < 0 ||
      o.m < 1 || o.m > kp::kMaxM || o.maxit < 0 || !(o.tol >= 0) || !(o.tol_seed >= 0))
    return kp::set_error(c, KP_ERR_ARG, "bad march options");
  kp_march_plan* P = new kp_march_plan();
  P->ctx = c;
  P->opt = o;
  P->groups.assign(groups, groups + ngroups);
  int nmaxS = 0, nmaxT = 0, wminS = 1 << 30, wminT = 1 << 30;
  for (int gi = 0; gi < ngroups; ++gi) {
    const kp_group& g = groups[gi];
    const int N = g.H * g.W;
    if (g.H < 1 || g.W < 1 || N > c->opt.max_n || g.nseed < 0 || g.ntgt < 0 ||
        (g.nseed && !g.m_seed) || (g.ntgt && !g.m_tgt) || (g.ntgt && !g.tgt_seed)) {
      kp_march_destroy(P);
      return kp::set_error(c, KP_ERR_ARG, "group %d: bad sizes or pointers", gi);
    }
    if (o.mode == KP_MARCH_PROJECTED || o.mode == KP_MARCH_GALERKIN || o.mode == KP_MARCH_LEARNED ||
        o.mode == KP_MARCH_LEARNED_ONLY)
      for (int t = 0; t < g.ntgt; ++t)
        if (g.tgt_seed[t] < 0 || g.tgt_seed[t] >= g.nseed) {
          kp_march_destroy(P);
          return kp::set_error(c, KP_ERR_ARG, "group %d target %d: seed index out of range", gi, t);
        }
    P->seed_off.push_back(P->seed_elems);
    P->tgt_off.push_back(P->tgt_elems);
    P->seed_elems += (size_t)g.nseed * N;
    P->tgt_elems += (size_t)g.ntgt * N;
    P->ns += g.nseed;
    P->nt += g.ntgt;
    if (g.nseed) { nmaxS = std::max(nmaxS, N); wminS = std::min(wminS, g.W); }
    if (g.ntgt) { nmaxT = std::max(nmaxT, N); wminT = std::min(wminT, g.W); }
  }
  if (2 * P->ns > c->opt.max_seeds) {
    kp_march_destroy(P);
    return kp::set_error(c, KP_ERR_ARG, "%d seeds need 2x%d basis slots (one set per timestep parity); max_seeds=%d",
                         P->ns, P->ns, c->opt.max_seeds);
  }
  P->mixed = c->opt.precision == KP_PREC_MIXED;
  kp_status s = KP_OK;
  if (P->ns) s = kp::gmres_shape(c, nmaxS, o.m_seed, &P->shS, P->mixed, wminS);
  if (s == KP_OK && P->nt) s = kp::gmres_shape(c, nmaxT, o.m, &P->shT, P->mixed, wminT);
  if (s == KP_OK && ((P->shS.cs && ngroups > 1) || (P->shT.cs && ngroups > 1))) {
    kp_march_destroy(P);
    return kp::set_error(c, KP_ERR_UNSUPPORTED, "grids above 4096 unknowns: one grid size per plan");
  }
  if (s != KP_OK) { kp_march_destroy(P); return s; }
  if (o.picard > 1 && (P->mixed || P->shT.cs || P->shS.cs)) {
    kp_march_destroy(P);
    return kp::set_error(c, KP_ERR_UNSUPPORTED, "Picard iterations need the FP64 one-block solver");
  }
  if (o.mode == KP_MARCH_GALERKIN && P->mixed) {
    // mixed precision: the Gram matrices on the tensor cores (kp_gram.cu) for
    // the one-block solver's grids (<= 4096 points)
    bool ok = !P->shT.cs && c->opt.max_a + 1 <= kp::kVbRows && c->opt.max_a <= kp::kMaxV;
    for (int gi = 0; gi < ngroups; ++gi) ok = ok && groups[gi].H * groups[gi].W <= 4096;
    if (!ok) {
      kp_march_destroy(P);
      return kp::set_error(c, KP_ERR_UNSUPPORTED, "mixed-precision exact Galerkin needs grids of <= 4096 points "
                           "(one-block solver) and max_a + 1 <= %d", kp::kVbRows);
    }
  } else if (o.mode == KP_MARCH_GALERKIN && P->shT.cs) {
    kp_march_destroy(P);
    return kp::set_error(c, KP_ERR_UNSUPPORTED, "exact Galerkin projection needs a one-block solver");
  }
  if (o.seed_solver != KP_SEED_GMRES &&
      (o.seed_solver != KP_SEED_BICGSTAB || P->mixed || P->shS.cs || P->shT.cs || o.picard > 1 ||
       o.m_seed < 4)) {
    kp_march_destroy(P);
    return kp::set_error(c, KP_ERR_UNSUPPORTED, "BiCGSTAB seeds need the FP64 one-block solver, "
                         "one Picard iteration and m_seed >= 4");
  }
  // seed cycling: predecessors in plan seed indices
  std::vector<int> cyc_prev(std::max(P->ns, 1), -1);
  {
    int base = 0;
    for (int gi = 0; gi < ngroups; ++gi) {
      const kp_group& g = groups[gi];
      for (int sidx = 0; sidx < g.nseed; ++sidx) {
        const int q = g.seed_prev ? g.seed_prev[sidx] : -1;
        if (q < -1 || q >= sidx) {
          kp_march_destroy(P);
          return kp::set_error(c, KP_ERR_ARG, "group %d seed %d: predecessor %d not in -1..%d", gi,
                               sidx, q, sidx - 1);
        }
        if (q >= 0) { cyc_prev[base + sidx] = base + q; P->cycling = true; }
      }
      base += g.nseed;
    }
  }
  if (P->cycling && (P->mixed || P->shS.cs || P->shT.cs)) {
    kp_march_destroy(P);
    return kp::set_error(c, KP_ERR_UNSUPPORTED, "seed cycling needs the FP64 one-block solver");
  }
  if (o.score && (P->mixed || P->shT.cs)) {
    kp_march_destroy(P);
    return kp::set_error(c, KP_ERR_UNSUPPORTED, "score extraction needs the FP64 one-block solver");
  }
  const bool learned = o.mode == KP_MARCH_LEARNED || o.mode == KP_MARCH_LEARNED_ONLY;
  if (learned) {
    if (!P->mixed || ngroups != 1 || o.picard > 1 || o.seed_solver != KP_SEED_GMRES || P->cycling ||
        !P->ns) {
      kp_march_destroy(P);
      return kp::set_error(c, KP_ERR_UNSUPPORTED, "learned march: mixed precision, one grid size, "
                           "GMRES seeds, one Picard iteration, no seed cycling");
    }
    if (!kp::cnn_march_ready(o.cnn, groups[0].H, groups[0].W)) {
      kp_march_destroy(P);
      return kp::set_error(c, KP_ERR_ARG, "learned march: needs a %dx%d network with 10 inputs, 1 output "
                           "and an inference batch", groups[0].H, groups[0].W);
    }
    P->cnn = o.cnn;
  }
  // window length: FP64 one-block solvers only; 2K slot sets must fit
  if (!P->mixed && !P->shS.cs && !P->shT.cs && o.window != 1 && P->nt > 0) {
    int K = o.window > 0 ? o.window : 8;
    if (P->ns) K = std::min(K, c->opt.max_seeds / (2 * P->ns));
    P->K = std::max(1, std::min(K, o.T));
  }
  cudaError_t e = cudaStreamCreateWithFlags(&P->st, cudaStreamNonBlocking);
  // the seed branch gets the higher priority: when both branches are ready
  // the block scheduler places the few seed blocks first and the persistent
  // target blocks take the remaining slots (and the seeds' once they finish)
  int prio_lo = 0, prio_hi = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&P->st2, cudaStreamNonBlocking, prio_hi);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P->join, cudaEventDisableTiming);
  const int ns = P->ns, nt = P->nt;
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = dmalloc(&P->S[k], P->seed_elems);
    if (e == cudaSuccess) e = dmalloc(&P->Tt[k], P->tgt_elems);
  }
  if (e == cudaSuccess) e = dmalloc(&P->g2, o.T);
  if (e == cudaSuccess) e = dmalloc(&P->step, 3);
  if (e == cudaSuccess) e = dmalloc(&P->err, 1);
  if (e == cudaSuccess) e = cudaMemset(P->err, 0, sizeof(int));
  // target classes (window mode with both small and larger grids: two)
  std::vector<int> cls_of(ngroups, 0);
  P->cls[0].sh = P->shT;
  P->cls[0].count = nt;
  if (P->K > 1 && nt > 0) {
    int nsmall = 0, nbig = 0;
    int nmaxA = 0, nmaxB = 0;
    double wA = 0, wB = 0;
    for (int gi = 0; gi < ngroups; ++gi) {
      const int N = groups[gi].H * groups[gi].W;
      if (!groups[gi].ntgt) continue;
      if (N <= 1024) { nsmall += groups[gi].ntgt; nmaxA = std::max(nmaxA, N); wA += (double)groups[gi].ntgt * N; }
      else { nbig += groups[gi].ntgt; nmaxB = std::max(nmaxB, N); wB += (double)groups[gi].ntgt * N; }
    }
    if (nsmall && nbig) {
      // larger grids first (class 0), launched with their share of the SMs;
      // the small-grid launch (class 1) takes the rest and the SMs they free
      P->ncls = 2;
      for (int gi = 0; gi < ngroups; ++gi) cls_of[gi] = groups[gi].H * groups[gi].W <= 1024 ? 1 : 0;
      kp_status s2 = kp::gmres_shape(c, nmaxB, o.m, &P->cls[0].sh, false, 0);
      if (s2 == KP_OK) s2 = kp::gmres_shape(c, nmaxA, o.m, &P->cls[1].sh, false, 0);
      if (s2 != KP_OK) { kp_march_destroy(P); return s2; }
      P->cls[0].first = 0;
      P->cls[0].count = nbig;
      P->cls[1].first = nbig;
      P->cls[1].count = nsmall;
      const int share = (int)(c->sms * wB / (wA + wB) + 0.5);
      P->cls[0].grid = std::max(1, std::min(std::min(nbig, c->sms - 1), share));
    }
    for (int ci = 0; ci < P->ncls; ++ci) {
      kp_march_plan::TClass& tc = P->cls[ci];
      const int per_sm = kp::gmres_fp64_blocks_per_sm(tc.sh.ept, tc.sh.nt, tc.sh.minb, tc.sh.smem);
      const int slots = (per_sm > 0 ? per_sm : 1) * c->sms;
      if (P->ncls == 1 || ci == 1) tc.grid = std::min(tc.count, o.target_blocks > 0 ? o.target_blocks : slots);
      tc.grid = std::max(1, tc.grid);
    }
  }
  if (e == cudaSuccess && P->K > 1) {
    e = dmalloc(&P->queue, 2);
    if (e == cudaSuccess) e = dmalloc(&P->done, nt);
  }
  if (e == cudaSuccess) e = dmalloc(&P->acc, o.T);
  if (e == cudaSuccess && P->cycling) {
    const size_t slots = (size_t)c->opt.max_seeds, a = (size_t)c->opt.max_a, n = (size_t)c->opt.max_n;
    e = dmalloc(&P->cyc_prev, (size_t)P->ns);
    if (e == cudaSuccess) e = dmalloc(&P->slotM, slots * n);
    if (e == cudaSuccess) e = dmalloc(&P->cycV, slots * (a + 1) * n);
    if (e == cudaSuccess) e = dmalloc(&P->cycR, slots * (a + 1) * a);
    if (e == cudaSuccess) e = dmalloc(&P->cycMeta, slots);
    if (e == cudaSuccess) e = dmalloc(&P->cycS, (size_t)P->K * P->ns * a * n);
    if (e == cudaSuccess)   // no slot is served before its first timestep
      e = cudaMemset(P->cycMeta, 0xff, slots * sizeof(kp::SlotMeta));
    if (e == cudaSuccess)
      e = cudaMemcpy(P->cyc_prev, cyc_prev.data(), (size_t)P->ns * sizeof(int), cudaMemcpyHostToDevice);
  }

  // one Krylov workspace per branch: seed blocks first, then target blocks
  size_t spS = 0, spT = 0;
  const int csS = P->shS.cs ? P->shS.cs : 1, csT = P->shT.cs ? P->shT.cs : 1;
  if (ns && P->shS.S < o.m_seed + 1) spS = (size_t)ns * csS * (o.m_seed + 1 - P->shS.S) * P->shS.ept * P->shS.nt;
  for (int ci = 0; ci < P->ncls; ++ci) {
    kp_march_plan::TClass& tc = P->cls[ci];
    tc.spill_off = spT;
    if (tc.count && tc.sh.S < o.m + 1)
      spT += (size_t)tc.count * csT * (o.m + 1 - tc.sh.S) * tc.sh.ept * tc.sh.nt;
  }
  if (e == cudaSuccess && spS + spT) {
    if (P->mixed) e = dmalloc(&P->spill32, spS + spT);
    else e = dmalloc(&P->spill, spS + spT);
  }
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = dmalloc(&P->desc[k], (size_t)ns + nt);
  if (e != cudaSuccess) {
    kp_status r = kp::cuda_error(c, e, "march allocation");
    kp_march_destroy(P);
    return r;
  }
  // descriptors for parity p: seeds of step n+1 (m_s^{n+1} in S[1-p] -> S[p]),
  // targets of step n (m_t^n in T[p] -> T[1-p]); b is the state itself, scaled by 1/dt
  const double dt = 1.0 / o.T;
  // internal target order: by seed within each group (stable)
  std::vector<int> hperm(std::max(nt, 1));
  {
    int base = 0;
    for (int gi = 0; gi < ngroups; ++gi) {
      const kp_group& g = groups[gi];
      P->tgt_base.push_back(base);
      std::vector<int> ord(g.ntgt);
      for (int k = 0; k < g.ntgt; ++k) ord[k] = k;
      if (o.mode == KP_MARCH_PROJECTED || o.mode == KP_MARCH_GALERKIN)
        std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return g.tgt_seed[x] < g.tgt_seed[y]; });
      for (int k = 0; k < g.ntgt; ++k) hperm[base + k] = ord[k];
      base += g.ntgt;
    }
  }
  if (e == cudaSuccess) e = dmalloc(&P->perm, nt);
  if (e == cudaSuccess) e = cudaMemcpy(P->perm, hperm.data(), nt * sizeof(int), cudaMemcpyHostToDevice);
  // first descriptor of each group's targets: class by class, groups in order
  std::vector<int> dfirst(ngroups, 0);
  {
    int q = 0;
    for (int ci = 0; ci < P->ncls; ++ci)
      for (int gi = 0; gi < ngroups; ++gi)
        if (cls_of[gi] == ci) { dfirst[gi] = q; q += groups[gi].ntgt; }
  }
  // score / embedding layout: groups in order, the caller's targets within a group
  std::vector<size_t> score_off(ngroups, 0);
  size_t score_stride = 0;
  for (int gi = 0; gi < ngroups; ++gi) {
    score_off[gi] = score_stride;
    score_stride += (size_t)groups[gi].ntgt * 2 * groups[gi].H * groups[gi].W;
  }
  P->score_stride = o.score ? score_stride : 0;
  for (int par = 0; par < 2 && e == cudaSuccess; ++par) {
    std::vector<SysDesc> hd((size_t)ns + nt);
    int si = 0, seed_base = 0;
    for (int gi = 0; gi < ngroups; ++gi) {
      const kp_group& g = groups[gi];
      const int N = g.H * g.W;
      for (int k = 0; k < g.nseed; ++k, ++si) {
        const size_t off = P->seed_off[gi] + (size_t)k * N;
        SysDesc d{};
        d.H = g.H; d.W = g.W; d.dt = dt; d.g2 = 0.0; d.h = 1.0 / g.H;
        d.mt = P->S[1 - par] + off;
        d.b = d.mt;
        d.x = P->S[par] + off;
        d.slot = 0;
        hd[si] = d;
      }
      for (int k = 0, ti = dfirst[gi]; k < g.ntgt; ++k, ++ti) {
        const size_t off = P->tgt_off[gi] + (size_t)k * N;
        SysDesc d{};
        d.H = g.H; d.W = g.W; d.dt = dt; d.g2 = 0.0; d.h = 1.0 / g.H;
        d.mt = P->Tt[par] + off;
        d.b = d.mt;
        d.x = P->Tt[1 - par] + off;
        const int u = hperm[P->tgt_base[gi] + k];   // user index of internal target k
        const int sd = (g.tgt_seed && g.tgt_seed[u] >= 0 && g.tgt_seed[u] < g.nseed) ? g.tgt_seed[u] : 0;
        d.slot = seed_base + sd;               // parity offset added on the device
        if (o.score) {
          d.score = o.score + score_off[gi] + (size_t)u * 2 * N;
          d.emb = o.embed + score_off[gi] + (size_t)u * 2 * N;
        }
        hd[(size_t)ns + ti] = d;
      }
      seed_base += g.nseed;
    }
    e = cudaMemcpy(P->desc[par], hd.data(), hd.size() * sizeof(SysDesc), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && P->cnn) {
      // learned guess tables: target k reads m^{n-1} (its descriptor's lagged
      // field) and the m_seed^n that the seeds of the previous launch wrote to
      // S[1 - par]; the network's output goes to gdelta, from which the
      // solver forms x_init
      std::vector<const double*> hp(nt), hs(nt);
      for (int k = 0; k < nt; ++k) {
        const SysDesc& d = hd[(size_t)ns + k];
        hp[k] = d.mt;
        hs[k] = P->S[1 - par] + (size_t)d.slot * groups[0].H * groups[0].W;
      }
      if (e == cudaSuccess && !P->gdelta) e = dmalloc(&P->gdelta, (size_t)nt * groups[0].H * groups[0].W);
      if (e == cudaSuccess && !P->grho) e = dmalloc(&P->grho, nt);
      if (e == cudaSuccess) e = dmalloc(&P->lg_prev[par], nt);
      if (e == cudaSuccess) e = dmalloc(&P->lg_seed[par], nt);
      if (e == cudaSuccess) e = cudaMemcpy(P->lg_prev[par], hp.data(), nt * sizeof(double*), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(P->lg_seed[par], hs.data(), nt * sizeof(double*), cudaMemcpyHostToDevice);
    }
  }
  if (e == cudaSuccess) e = cudaMemcpy(P->g2, o.g2, o.T * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && P->mixed && (o.mode == KP_MARCH_PROJECTED || o.mode == KP_MARCH_GALERKIN) && ns > 0 &&
      nt > 0 && c->opt.max_a + 1 <= kp::kVbRows) {
    // tensor-core projection: BF16 right-hand sides, c = V^T b, tile lists
    const int vb_ld = c->vb_ld;
    e = dmalloc(&P->Bb, (size_t)nt * vb_ld);
    if (e == cudaSuccess) e = cudaMemset(P->Bb, 0, (size_t)nt * vb_ld * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = dmalloc(&P->Cp, (size_t)nt * kp::kVbRows);
    std::vector<kp::ProjTile> tl[2];
    int seed_base = 0;
    P->mapB.resize(ngroups);
    P->mapV.resize(ngroups);
    for (int gi = 0; gi < ngroups && e == cudaSuccess; ++gi) {
      const kp_group& g = groups[gi];
      const int N = g.H * g.W;
      P->tile_off.push_back((int)tl[0].size());
      int k = 0;
      while (k < g.ntgt) {                      // runs of targets sharing a seed
        const int sd = g.tgt_seed[hperm[P->tgt_base[gi] + k]];
        int end = k;
        while (end < g.ntgt && g.tgt_seed[hperm[P->tgt_base[gi] + end]] == sd) ++end;
        for (int q = k; q < end; q += 128)
          for (int par = 0; par < 2; ++par) {
            kp::ProjTile t;
            t.row0 = q;
            t.vrow0 = (par * ns + seed_base + sd) * kp::kVbRows;
            t.crow0 = P->tgt_base[gi] + q;
            t.count = std::min(128, end - q);
            t.nv = kp::kVbRows;
            t.ccol0 = 0;
            t.kc0 = t.kc1 = 0;
            t.atomic = 0;
            tl[par].push_back(t);
          }
        k = end;
      }
      P->tile_cnt.push_back((int)tl[0].size() - P->tile_off.back());
      if (g.ntgt) e = kp::make_bf16_map(&P->mapB[gi], P->Bb + (size_t)P->tgt_base[gi] * vb_ld,
                                        g.ntgt, N, vb_ld, 128);
      if (e == cudaSuccess)
        e = kp::make_bf16_map(&P->mapV[gi], c->slotVb, c->opt.max_seeds * kp::kVbRows, N, vb_ld,
                              kp::kVbRows);
      seed_base += g.nseed;
    }
    for (int par = 0; par < 2 && e == cudaSuccess; ++par) {
      e = dmalloc(&P->tiles[par], tl[par].size());
      if (e == cudaSuccess)
        e = cudaMemcpy(P->tiles[par], tl[par].data(), tl[par].size() * sizeof(kp::ProjTile),
                       cudaMemcpyHostToDevice);
    }
    P->gemm_grid = c->sms;
  }
  if (e == cudaSuccess && P->mixed && o.mode == KP_MARCH_GALERKIN && ns > 0 && nt > 0) {
    // Gram matrices: product rows of the seed bases (pairs p * A + q, both
    // slot sets), coefficient rows of the targets, C = Q P^T tiles per run of
    // targets sharing a seed and per 48 pairs
    const int A = c->opt.max_a;
    int nmax = 0;
    for (int gi = 0; gi < ngroups; ++gi) nmax = std::max(nmax, groups[gi].H * groups[gi].W);
    P->gram_A = A;
    P->p_ld = P->q_ld = (2 * nmax + 7) / 8 * 8;
    const size_t pairs = (size_t)A * A;
    e = dmalloc(&P->Pb, (size_t)2 * ns * pairs * P->p_ld);
    if (e == cudaSuccess) e = cudaMemset(P->Pb, 0, (size_t)2 * ns * pairs * P->p_ld * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = dmalloc(&P->G0, (size_t)2 * ns * pairs);
    if (e == cudaSuccess) e = dmalloc(&P->Qb, (size_t)nt * P->q_ld);
    if (e == cudaSuccess) e = cudaMemset(P->Qb, 0, (size_t)nt * P->q_ld * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = dmalloc(&P->Cg, (size_t)nt * pairs);
    std::vector<kp::ProjTile> tl[2];
    int seed_base = 0;
    P->mapQ.resize(ngroups);
    P->mapP.resize(ngroups);
    for (int gi = 0; gi < ngroups && e == cudaSuccess; ++gi) {
      const kp_group& g = groups[gi];
      const int K2 = 2 * g.H * g.W;
      P->gtile_off.push_back((int)tl[0].size());
      int k = 0;
      while (k < g.ntgt) {
        const int sd = g.tgt_seed[hperm[P->tgt_base[gi] + k]];
        int end = k;
        while (end < g.ntgt && g.tgt_seed[hperm[P->tgt_base[gi] + end]] == sd) ++end;
        for (int q = k; q < end; q += 128)
          for (int pb = 0; pb < (int)pairs; pb += 48)
            for (int par = 0; par < 2; ++par) {
              kp::ProjTile t;
              t.row0 = q;
              t.vrow0 = (int)((size_t)(par * ns + seed_base + sd) * pairs) + pb;
              t.crow0 = P->tgt_base[gi] + q;
              t.count = std::min(128, end - q);
              t.nv = std::min(48, (int)pairs - pb);
              t.ccol0 = pb;
              t.kc0 = t.kc1 = 0;
              t.atomic = 0;
              tl[par].push_back(t);
            }
        k = end;
      }
      P->gtile_cnt.push_back((int)tl[0].size() - P->gtile_off.back());
      if (g.ntgt) e = kp::make_bf16_map(&P->mapQ[gi], P->Qb + (size_t)P->tgt_base[gi] * P->q_ld, g.ntgt, K2,
                                        P->q_ld, 128);
      if (e == cudaSuccess)
        e = kp::make_bf16_map(&P->mapP[gi], P->Pb, (int)(2 * ns * pairs), K2, P->p_ld, 48);
      seed_base += g.nseed;
    }
    for (int par = 0; par < 2 && e == cudaSuccess; ++par) {
      e = dmalloc(&P->gtiles[par], tl[par].size());
      if (e == cudaSuccess)
        e = cudaMemcpy(P->gtiles[par], tl[par].data(), tl[par].size() * sizeof(kp::ProjTile),
                       cudaMemcpyHostToDevice);
    }
    P->gemm_grid = c->sms;
  }
  if (e != cudaSuccess) {
    kp_status r = kp::cuda_error(c, e, "march tables");
    kp_march_destroy(P);
    return r;
  }
  if (o.use_graph && P->K > 1) {
    cudaGraph_t gr = nullptr;
    e = cudaStreamBeginCapture(P->st, cudaStreamCaptureModeThreadLocal);
    kp_status r = KP_OK;
    if (e == cudaSuccess) {
      r = enqueue_window(P, nullptr, &P->launches_per_step);
      cudaError_t e2 = cudaStreamEndCapture(P->st, &gr);
      if (r == KP_OK) e = e2;
    }
    if (r == KP_OK && e == cudaSuccess) e = cudaGraphInstantiate(&P->graph[0], gr, 0);
    if (gr) cudaGraphDestroy(gr);
    if (r != KP_OK || e != cudaSuccess) {
      if (r == KP_OK) r = kp::cuda_error(c, e, "march graph capture");
      kp_march_destroy(P);
      return r;
    }
  } else if (o.use_graph) {
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
  const int q0 = n0 & 1;
  cudaError_t e = cudaSuccess;
  // after the caller's stream: states in, counters and totals reset
  cudaEvent_t sync_ev = nullptr;
  e = cudaEventCreateWithFlags(&sync_ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(sync_ev, c->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(P->st, sync_ev, 0);
  for (size_t gi = 0; gi < P->groups.size() && e == cudaSuccess; ++gi) {
    const kp_group& g = P->groups[gi];
    const size_t N = (size_t)g.H * g.W;
    if (g.nseed) e = cudaMemcpyAsync(P->S[q0] + P->seed_off[gi], g.m_seed, g.nseed * N * sizeof(double), cudaMemcpyDeviceToDevice, P->st);
    if (e == cudaSuccess && g.ntgt)
      e = kp::launch_permute(P->Tt[q0] + P->tgt_off[gi], g.m_tgt, P->perm + P->tgt_base[gi], g.ntgt,
                             (int)N, 1, P->st);
    if (e == cudaSuccess && g.ntgt && P->Bb)
      e = kp::launch_to_bf16(P->Bb + (size_t)P->tgt_base[gi] * c->vb_ld, c->vb_ld,
                             P->Tt[q0] + P->tgt_off[gi], g.ntgt, (int)N, 1.0, P->st);   // b as stored
  }
  P->host_step[0] = n0;
  P->host_step[1] = n0 + steps;
  P->host_step[2] = n0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(P->step, P->host_step, 3 * sizeof(int), cudaMemcpyHostToDevice, P->st);
  if (e == cudaSuccess && P->done) e = cudaMemsetAsync(P->done, 0, (size_t)P->nt * sizeof(int), P->st);
  if (e == cudaSuccess && P->queue) e = cudaMemsetAsync(P->queue, 0, 2 * sizeof(int), P->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->acc + n0, 0, (size_t)steps * sizeof(kp::StepAcc), P->st);
  std::vector<cudaEvent_t> ev;
  int launches = 0;
  const int K = P->K;
  const int nwin = (steps + K - 1) / K;       // launches of the step (K = 1) or window graph
  constexpr int kEv = 6;                      // events per step or window (see enqueue_step)
  if (e == cudaSuccess && timing) {
    ev.resize((size_t)nwin * kEv + 2, nullptr);
    for (auto& x : ev)
      if (e == cudaSuccess) e = cudaEventCreate(&x);
  }
  kp_status r = KP_OK;
  // prologue: seeds of step n0 (or of the first window), whose bases serve
  // the first targets
  if (e == cudaSuccess && P->ns) {
    kp::GmresParams g = solver_params(P, true, 1 - q0, 0);
    if (timing) e = cudaEventRecord(ev[(size_t)nwin * kEv], P->st);
    if (e == cudaSuccess) e = launch_solver(P, g, P->shS, P->st);
    ++launches;
    if (P->cycling && e == cudaSuccess) { e = launch_cycle(P, 0, P->st); ++launches; }
    if (timing && e == cudaSuccess) e = cudaEventRecord(ev[(size_t)nwin * kEv + 1], P->st);
  }
  for (int k = 0; k < nwin && e == cudaSuccess && r == KP_OK; ++k) {
    const int par = K > 1 ? 0 : (n0 + k) & 1;
    if (timing) {
      int nl = 0;
      r = K > 1 ? enqueue_window(P, ev.data() + (size_t)k * kEv, &nl)
                : enqueue_step(P, par, ev.data() + (size_t)k * kEv, &nl);
      launches += nl;
    } else if (P->graph[par]) {
      e = cudaGraphLaunch(P->graph[par], P->st);
      launches += P->launches_per_step;
    } else {
      int nl = 0;
      r = K > 1 ? enqueue_window(P, nullptr, &nl) : enqueue_step(P, par, nullptr, &nl);
      launches += nl;
    }
  }
  const int fin = (n0 + steps) & 1;
  for (size_t gi = 0; gi < P->groups.size() && e == cudaSuccess && r == KP_OK; ++gi) {
    const kp_group& g = P->groups[gi];
    const size_t N = (size_t)g.H * g.W;
    if (g.nseed) e = cudaMemcpyAsync(g.m_seed, P->S[fin] + P->seed_off[gi], g.nseed * N * sizeof(double), cudaMemcpyDeviceToDevice, P->st);
    if (e == cudaSuccess && g.ntgt)
      e = kp::launch_permute(g.m_tgt, P->Tt[fin] + P->tgt_off[gi], P->perm + P->tgt_base[gi], g.ntgt,
                             (int)N, 0, P->st);
  }
  if (e == cudaSuccess) e = cudaEventRecord(sync_ev, P->st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(c->stream, sync_ev, 0);
  if (e == cudaSuccess && (stats || timing)) e = cudaStreamSynchronize(P->st);
  if (e == cudaSuccess && stats) {
    std::vector<kp::StepAcc> h(steps);
    e = cudaMemcpy(h.data(), P->acc + n0, steps * sizeof(kp::StepAcc), cudaMemcpyDeviceToHost);
    for (int k = 0; k < steps && e == cudaSuccess; ++k) {
      const kp::StepAcc& a = h[k];
      double mr;
      std::memcpy(&mr, &a.max_res_bits, sizeof(mr));
      stats[k].seed_iters = (double)a.seed_iters;
      stats[k].tgt_iters = (double)a.tgt_iters;
      stats[k].tgt_iters_max = (double)a.tgt_max_iters;
      stats[k].not_converged = (double)a.not_converged;
      stats[k].max_rel_res = mr;
      stats[k].refine_flops = (double)a.tgt_flops;
      stats[k].seed_flops = (double)a.seed_flops;
      stats[k].proj_flops = (double)a.proj_flops;
      stats[k].refine_flops32 = (double)a.tgt_flops32;
    }
  }
  if (e == cudaSuccess && (stats || timing)) {
    int herr = 0;
    e = cudaMemcpy(&herr, P->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && herr) {
      cudaMemset(P->err, 0, sizeof(int));
      r = kp::set_error(c, KP_ERR_TIMEOUT, "march: a device wait gave up (flags 0x%x)", herr);
    }
  }
  if (e == cudaSuccess && timing) {
    std::memset(timing, 0, sizeof(*timing));
    float t = 0.f;
    if (P->ns) {
      e = cudaEventElapsedTime(&t, ev[(size_t)nwin * kEv], ev[(size_t)nwin * kEv + 1]);
      timing->seed_ms += t;
    }
    for (int k = 0; k < nwin && e == cudaSuccess; ++k) {
      cudaEvent_t* x = ev.data() + (size_t)k * kEv;
      if (P->cnn && P->nt) {
        e = cudaEventElapsedTime(&t, x[4], x[5]);
        timing->proj_ms += t;
      }
      if (P->ns) {
        e = cudaEventElapsedTime(&t, x[0], x[1]);
        timing->seed_ms += t;
      }
      if (e == cudaSuccess && P->nt) {
        e = cudaEventElapsedTime(&t, x[2], x[3]);
        timing->refine_ms += t;
      }
    }
    if (e == cudaSuccess && P->ns && P->nt)
      e = cudaEventElapsedTime(&timing->step_ms, ev[(size_t)nwin * kEv], ev[(size_t)(nwin - 1) * kEv + 3]);
  }
  if (timing) timing->launches = launches;
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  if (sync_ev) cudaEventDestroy(sync_ev);
  if (r != KP_OK) return r;
  return e == cudaSuccess ? KP_OK : kp::cuda_error(c, e, "march run");
}

}  // extern "C"
