// kp_gmres.cu -- batched restarted GMRES(m) for the five-point Fokker-Planck
// systems of Sec. 2.3 (Eq. 11-13), FP64, one thread block per system.
//
// GB300 design notes (FP64 runs at 1/64 of the FP32 rate on this part, about
// 2 FP64 FMA per clock per SM, so FP64 instructions -- not HBM bytes -- bound
// this kernel):
//  * The operator is applied matrix-free.  Each thread keeps the four
//    off-diagonal coefficients of its EPT grid points in registers (computed
//    once per solve from the lagged field m~), the diagonal is a scalar, and
//    out-of-grid neighbours get a zero coefficient and a clamped index, so the
//    stencil is 1 MUL + 4 FMA per point with no branches.
//  * Krylov vectors v_0..v_{S-1} live in shared memory; the stencil reads its
//    neighbours there.  Vectors beyond S go to a per-block device workspace.
//  * Orthogonalisation is classical Gram-Schmidt applied twice (CGS2): every
//    pass is one batched reduction of all <v_i, w> at once instead of j
//    sequential reductions.  Reductions are warp reduce-scatter butterflies
//    over 8 values (about one FP64 add per value per lane instead of five)
//    followed by one cross-warp sum.
//  * Hessenberg, Givens rotations and the least-squares solve stay in FP64 on
//    one lane; the true residual b - A x is recomputed in FP64 at every restart.
#include "kp_internal.cuh"

namespace kp {
namespace {

struct Smem {
  double* V;     // [S][npad]
  double* xs;    // [npad]
  double* red;   // [NWARPS][kMaxV]
  double* hb;    // [kMaxV]
  double* Hr;    // [(m+1) * m] rotated Hessenberg, column-major, ld m+1
  double* g;     // [m+1]
  double* cs;    // [m]
  double* sn;    // [m]
  double* y;     // [m]
  double* sc;    // [8] scalars
  int* fl;       // [8] flags
};

__device__ __forceinline__ Smem carve(double* base, int S, int npad, int nwarps, int m) {
  Smem s;
  s.V = base;
  s.xs = s.V + (size_t)S * npad;
  s.red = s.xs + npad;
  s.hb = s.red + nwarps * kMaxV;
  s.Hr = s.hb + kMaxV;
  s.g = s.Hr + (m + 1) * m;
  s.cs = s.g + (m + 1);
  s.sn = s.cs + m;
  s.y = s.sn + m;
  s.sc = s.y + m;
  s.fl = reinterpret_cast<int*>(s.sc + 8);
  return s;
}

// Givens rotation [c s; -s c] [a; b] = [r; 0].
__device__ __forceinline__ void givens(double a, double b, double& c, double& s) {
  if (b == 0.0) { c = 1.0; s = 0.0; return; }
  const double r = hypot(a, b);
  const double ir = 1.0 / r;
  c = a * ir;
  s = b * ir;
}

template <int EPT, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) gmres_fp64_kernel(const GmresParams p) {
  constexpr int NWARPS = NT / 32;
  extern __shared__ __align__(16) double smem_raw[];
  const int npad = EPT * NT;
  const int m = p.m;
  const int ld = m + 1;
  Smem sm = carve(smem_raw, p.S, npad, NWARPS, m);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  double* spill = p.spill ? p.spill + (size_t)blockIdx.x * (m + 1 - p.S) * npad : nullptr;
  auto slot = [&](int i) -> double* {
    return i < p.S ? sm.V + (size_t)i * npad : spill + (size_t)(i - p.S) * npad;
  };

  for (int sysi = blockIdx.x; sysi < p.nsys; sysi += gridDim.x) {
    const SysDesc d = p.sys[sysi];
    const int H = d.H, W = d.W, N = H * W;
    const double hh = d.h;
    const double g2 = p.step ? p.g2_sched[*p.step] : d.g2;
    const double cc = g2 / (2.0 * hh * hh);
    const double ee = g2 / (8.0 * hh * hh);
    const double cd = 1.0 / d.dt + 2.0 * g2 / (hh * hh);
    const double i2h = 1.0 / (2.0 * hh);
    const bool capture = p.capV != nullptr;
    double* capV = capture ? p.capV + (size_t)sysi * (p.cap_a + 1) * p.cap_ld : nullptr;
    double* capH = capture ? p.capH + (size_t)sysi * (p.cap_a + 1) * p.cap_a : nullptr;

    // stencil coefficients (Sec. 2.3, listing after Eq. 11); zero where the
    // neighbour lies outside the grid
    double cE[EPT], cW[EPT], cN[EPT], cS[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int pp = tid + k * NT;
      cE[k] = cW[k] = cN[k] = cS[k] = 0.0;
      if (pp < N) {
        const int i = pp / H, j = pp - i * H;
        const double mE = (i + 1 < W) ? d.mt[pp + H] : 0.0;
        const double mW = (i > 0) ? d.mt[pp - H] : 0.0;
        const double mN = (j + 1 < H) ? d.mt[pp + 1] : 0.0;
        const double mS = (j > 0) ? d.mt[pp - 1] : 0.0;
        const double fxp = d.fx ? d.fx[pp] : 0.0;
        const double fyp = d.fy ? d.fy[pp] : 0.0;
        const double dmx = mE - mW, dmy = mN - mS;
        if (i + 1 < W) cE[k] = -cc + fxp * i2h - ee * dmx;
        if (i > 0) cW[k] = -cc - fxp * i2h + ee * dmx;
        if (j + 1 < H) cN[k] = -cc + fyp * i2h - ee * dmy;
        if (j > 0) cS[k] = -cc - fyp * i2h + ee * dmy;
      }
    }
    auto apply = [&](const double* v, double (&out)[EPT]) {
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int pp = tid + k * NT;
        if (pp < N) {
          const int pe = min(pp + H, N - 1), pw = max(pp - H, 0);
          const int pn = min(pp + 1, N - 1), ps = max(pp - 1, 0);
          out[k] = cd * v[pp] + cE[k] * v[pe] + cW[k] * v[pw] + cN[k] * v[pn] + cS[k] * v[ps];
        } else {
          out[k] = 0.0;
        }
      }
    };

    // x -> shared memory; r = b - A x; ||b||, ||r||
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int pp = tid + k * NT;
      sm.xs[pp] = (pp < N) ? d.x[pp] : 0.0;
    }
    __syncthreads();
    double w[EPT];
    auto residual = [&]() {
      apply(sm.xs, w);
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int pp = tid + k * NT;
        w[k] = (pp < N) ? d.b[pp] - w[k] : 0.0;
      }
    };
    residual();
    block_partials<NT>(2, [&](int i) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int pp = tid + k * NT;
        const double bv = (pp < N) ? d.b[pp] : 0.0;
        s += (i == 0) ? bv * bv : w[k] * w[k];
      }
      return s;
    }, sm.red);
    if (tid == 0) {
      sm.sc[0] = sqrt(cross_warp<NT>(sm.red, 0));
      sm.sc[1] = sqrt(cross_warp<NT>(sm.red, 1));
    }
    __syncthreads();
    const double bnorm = sm.sc[0];
    double beta = sm.sc[1];

    int steps = 0, status = KP_NOT_CONVERGED, cycle = 0;
    if (bnorm == 0.0) {
#pragma unroll
      for (int k = 0; k < EPT; ++k) sm.xs[tid + k * NT] = 0.0;
      beta = 0.0;
      status = KP_OK;
    }
    while (status == KP_NOT_CONVERGED) {
      if (beta <= p.tol * bnorm) { status = KP_OK; break; }
      if (!isfinite(beta)) { status = KP_BREAKDOWN; break; }
      if (steps >= p.maxit) break;
      {
        const double ib = 1.0 / beta;
        double* v0 = slot(0);
#pragma unroll
        for (int k = 0; k < EPT; ++k) {
          const int pp = tid + k * NT;
          v0[pp] = w[k] * ib;
          if (capture && cycle == 0 && pp < N) capV[pp] = w[k] * ib;
        }
        if (tid == 0) sm.g[0] = beta;
      }
      int kdone = 0;
      int brk = 0;
      for (int j = 0; j < m; ++j) {
        __syncthreads();                       // v_j complete
        apply(slot(j), w);
        ++steps;
        const int nh = j + 1;
        auto dots = [&](int i) {
          double s = 0.0;
          if (i < nh) {
            const double* vi = slot(i);
#pragma unroll
            for (int k = 0; k < EPT; ++k) s += vi[tid + k * NT] * w[k];
          } else {
#pragma unroll
            for (int k = 0; k < EPT; ++k) s += w[k] * w[k];
          }
          return s;
        };
        // CGS pass 1: h_i = <v_i, w>, plus ||w||^2 before orthogonalisation
        block_partials<NT>(nh + 1, dots, sm.red);
        if (warp == 0) {
          double sq = 0.0;
          for (int i = lane; i <= nh; i += 32) {
            const double s = cross_warp<NT>(sm.red, i);
            sm.hb[i] = s;
            if (i < nh) { sm.Hr[i + j * ld] = s; sq += s * s; }
          }
          sq = warp_sum(sq);
          if (lane == 0) {
            const double ww0 = sm.hb[nh];
            sm.sc[2] = ww0;
            // DGKS: a second pass only if the first removed over half the norm^2
            sm.fl[0] = (p.reorth == 0) || (ww0 - sq < 0.5 * ww0);
          }
        }
        __syncthreads();
        for (int i = 0; i < nh; ++i) {
          const double hi = sm.hb[i];
          const double* vi = slot(i);
#pragma unroll
          for (int k = 0; k < EPT; ++k) w[k] = fma(-hi, vi[tid + k * NT], w[k]);
        }
        if (sm.fl[0]) {
          // CGS pass 2 (reorthogonalisation)
          block_partials<NT>(nh, dots, sm.red);
          if (warp == 0) {
            for (int i = lane; i < nh; i += 32) {
              const double s = cross_warp<NT>(sm.red, i);
              sm.hb[i] = s;
              sm.Hr[i + j * ld] += s;
            }
          }
          __syncthreads();
          for (int i = 0; i < nh; ++i) {
            const double hi = sm.hb[i];
            const double* vi = slot(i);
#pragma unroll
            for (int k = 0; k < EPT; ++k) w[k] = fma(-hi, vi[tid + k * NT], w[k]);
          }
        }
        // ||w|| after orthogonalisation, then Givens update of column j
        block_partials<NT>(1, [&](int) {
          double s = 0.0;
#pragma unroll
          for (int k = 0; k < EPT; ++k) s += w[k] * w[k];
          return s;
        }, sm.red);
        if (tid == 0) {
          const double hn = sqrt(cross_warp<NT>(sm.red, 0));
          const int b = !(hn > 1e-14 * sqrt(sm.sc[2]));
          sm.Hr[(j + 1) + j * ld] = hn;
          if (capture && cycle == 0 && j < p.cap_a) {
            for (int i = 0; i <= j + 1; ++i) capH[i + j * (p.cap_a + 1)] = sm.Hr[i + j * ld];
          }
          for (int i = 0; i < j; ++i) {
            const double t1 = sm.Hr[i + j * ld], t2 = sm.Hr[(i + 1) + j * ld];
            sm.Hr[i + j * ld] = sm.cs[i] * t1 + sm.sn[i] * t2;
            sm.Hr[(i + 1) + j * ld] = -sm.sn[i] * t1 + sm.cs[i] * t2;
          }
          double c, s;
          givens(sm.Hr[j + j * ld], sm.Hr[(j + 1) + j * ld], c, s);
          sm.cs[j] = c;
          sm.sn[j] = s;
          sm.Hr[j + j * ld] = c * sm.Hr[j + j * ld] + s * sm.Hr[(j + 1) + j * ld];
          sm.Hr[(j + 1) + j * ld] = 0.0;
          sm.g[j + 1] = -s * sm.g[j];
          sm.g[j] = c * sm.g[j];
          const double res = fabs(sm.g[j + 1]);
          sm.sc[3] = hn;
          sm.fl[1] = b;
          sm.fl[2] = (res <= p.tol * bnorm) || b || (steps >= p.maxit) || (j + 1 == m);
        }
        __syncthreads();
        brk = sm.fl[1];
        kdone = j + 1;
        if (!brk) {
          const double ih = 1.0 / sm.sc[3];
          double* vn = slot(j + 1);
#pragma unroll
          for (int k = 0; k < EPT; ++k) {
            const int pp = tid + k * NT;
            vn[pp] = w[k] * ih;
            if (capture && cycle == 0 && j + 1 <= p.cap_a && pp < N)
              capV[(size_t)(j + 1) * p.cap_ld + pp] = w[k] * ih;
          }
        }
        if (sm.fl[2]) break;
      }
      // y = R^{-1} g (back substitution, one lane)
      if (tid == 0) {
        for (int i = kdone - 1; i >= 0; --i) {
          double s = sm.g[i];
          for (int l = i + 1; l < kdone; ++l) s -= sm.Hr[i + l * ld] * sm.y[l];
          sm.y[i] = s / sm.Hr[i + i * ld];
        }
        if (capture && cycle == 0) {
          const int a = kdone < p.cap_a ? kdone : p.cap_a;
          p.capMeta[sysi].a = a;
          p.capMeta[sysi].has_next = (a < kdone) || !brk;
          p.capMeta[sysi].N = N;
          p.capMeta[sysi].valid = 1;
        }
      }
      __syncthreads();
      for (int i = 0; i < kdone; ++i) {
        const double yi = sm.y[i];
        const double* vi = slot(i);
#pragma unroll
        for (int k = 0; k < EPT; ++k) sm.xs[tid + k * NT] = fma(yi, vi[tid + k * NT], sm.xs[tid + k * NT]);
      }
      __syncthreads();
      residual();                              // true FP64 residual
      block_partials<NT>(1, [&](int) {
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < EPT; ++k) s += w[k] * w[k];
        return s;
      }, sm.red);
      if (tid == 0) sm.sc[1] = sqrt(cross_warp<NT>(sm.red, 0));
      __syncthreads();
      beta = sm.sc[1];
      ++cycle;
    }
    if (capture && cycle == 0 && tid == 0) {   // converged before any step
      p.capMeta[sysi].a = 0;
      p.capMeta[sysi].has_next = 0;
      p.capMeta[sysi].N = N;
      p.capMeta[sysi].valid = 1;
    }
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int pp = tid + k * NT;
      if (pp < N) d.x[pp] = sm.xs[pp];
    }
    if (tid == 0 && p.info) {
      kp_info inf;
      inf.iters = steps;
      inf.status = status;
      inf.rel_res = bnorm > 0.0 ? beta / bnorm : 0.0;
      p.info[sysi] = inf;
    }
    __syncthreads();                           // shared memory reused by the next system
  }
}

// y = A x (mode 0) or b = m^{n-1}/dt - Div_h f (mode 1), one block per system.
__global__ void apply_rhs_kernel(const SysDesc* sys, int nsys, int mode) {
  const SysDesc d = sys[blockIdx.x];
  const int H = d.H, W = d.W, N = H * W;
  const double hh = d.h;
  const double cc = d.g2 / (2.0 * hh * hh);
  const double ee = d.g2 / (8.0 * hh * hh);
  const double cd = 1.0 / d.dt + 2.0 * d.g2 / (hh * hh);
  const double i2h = 1.0 / (2.0 * hh);
  for (int pp = threadIdx.x; pp < N; pp += blockDim.x) {
    const int i = pp / H, j = pp - i * H;
    if (mode == 1) {
      const double fE = (d.fx && i + 1 < W) ? d.fx[pp + H] : 0.0;
      const double fW = (d.fx && i > 0) ? d.fx[pp - H] : 0.0;
      const double fN = (d.fy && j + 1 < H) ? d.fy[pp + 1] : 0.0;
      const double fS = (d.fy && j > 0) ? d.fy[pp - 1] : 0.0;
      d.x[pp] = d.b[pp] / d.dt - ((fE - fW) + (fN - fS)) * i2h;
      continue;
    }
    const double mE = (i + 1 < W) ? d.mt[pp + H] : 0.0;
    const double mW = (i > 0) ? d.mt[pp - H] : 0.0;
    const double mN = (j + 1 < H) ? d.mt[pp + 1] : 0.0;
    const double mS = (j > 0) ? d.mt[pp - 1] : 0.0;
    const double fxp = d.fx ? d.fx[pp] : 0.0;
    const double fyp = d.fy ? d.fy[pp] : 0.0;
    const double dmx = mE - mW, dmy = mN - mS;
    double y = cd * d.b[pp];
    if (i + 1 < W) y += (-cc + fxp * i2h - ee * dmx) * d.b[pp + H];
    if (i > 0) y += (-cc - fxp * i2h + ee * dmx) * d.b[pp - H];
    if (j + 1 < H) y += (-cc + fyp * i2h - ee * dmy) * d.b[pp + 1];
    if (j > 0) y += (-cc - fyp * i2h + ee * dmy) * d.b[pp - 1];
    d.x[pp] = y;
  }
}

}  // namespace

size_t gmres_fp64_smem_bytes(int ept, int nt, int S, int m) {
  const int npad = ept * nt;
  const size_t doubles = (size_t)S * npad + npad + (nt / 32) * kMaxV + kMaxV +
                         (size_t)(m + 1) * m + (m + 1) + 3 * m + 8;
  return doubles * sizeof(double) + 8 * sizeof(int);
}

template <int EPT, int NT, int MINB>
static cudaError_t launch_one(const GmresParams& p, size_t smem, cudaStream_t st) {
  auto k = gmres_fp64_kernel<EPT, NT, MINB>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<p.nsys, NT, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_gmres_fp64(const GmresParams& p, int ept, int nt, size_t smem,
                              cudaStream_t st) {
  if (ept == 4 && nt == 256) return launch_one<4, 256, 2>(p, smem, st);
  if (ept == 8 && nt == 512) return launch_one<8, 512, 1>(p, smem, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_gmres_fp64_1k_grid(const GmresParams& p, size_t smem, int grid,
                                      cudaStream_t st) {
  auto k = gmres_fp64_kernel<4, 256, 2>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, 256, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_apply(const SysDesc* sys, int nsys, int mode, cudaStream_t st) {
  apply_rhs_kernel<<<nsys, 256, 0, st>>>(sys, nsys, mode);
  return cudaGetLastError();
}

}  // namespace kp
