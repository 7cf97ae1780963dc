// kp_project.cu -- the seed-basis store and the Galerkin projection of
// Sec. 3, Phase 2, in FP64:
//   store:    V_a^n and the Givens QR factors of H_a = V_a^T A_seed V_a
//             (taken from the seed's Arnoldi process), once per seed;
//   project:  c = V_a^T r,  alpha = H_a^{-1} c,  x <- x + V_a alpha,
//             one thread block per target, the seed's V read through L2 by
//             all targets that share it.
#include "kp_internal.cuh"

namespace kp {
namespace {

// Copies the captured basis of system p.sys into slot p.seed_id and factors
// its Hessenberg matrix.  One block; thread 0 does the (tiny) factorisation.
__global__ void factor_kernel(FactorParams p) {
  p.sys += blockIdx.x;
  p.seed_id += blockIdx.x;
  if (p.step) p.timestep = *p.step;
  const CapMeta cm = p.capMeta[p.sys];
  const int a = cm.valid ? cm.a : 0;
  const int hn = cm.valid ? cm.has_next : 0;
  const int N = cm.N;
  const double* cv = p.capV + (size_t)p.sys * (p.cap_a + 1) * p.cap_ld;
  double* sv = p.slotV + (size_t)p.seed_id * (p.max_a + 1) * p.ld;
  const int nvec = a + hn;
  if (p.capV32) {
    const float* cv32 = p.capV32 + (size_t)p.sys * (p.cap_a + 1) * p.cap_ld;
    float* sv32 = p.slotV32 + (size_t)p.seed_id * (p.max_a + 1) * p.ld;
    for (int idx = threadIdx.x; idx < nvec * N; idx += blockDim.x) {
      const int k = idx / N, q = idx - k * N;
      sv32[(size_t)k * p.ld + q] = cv32[(size_t)k * p.cap_ld + q];
    }
  } else {
    for (int idx = threadIdx.x; idx < nvec * N; idx += blockDim.x) {
      const int k = idx / N, q = idx - k * N;
      sv[(size_t)k * p.ld + q] = cv[(size_t)k * p.cap_ld + q];
    }
  }
  if (threadIdx.x != 0) return;
  const int cld = p.cap_a + 1;
  const int sld = p.max_a + 1;
  const double* ch = p.capH + (size_t)p.sys * cld * p.cap_a;
  double* sh = p.slotH + (size_t)p.seed_id * sld * p.max_a;
  double* R = p.slotR + (size_t)p.seed_id * sld * p.max_a;   // (a+1) x a, ld max_a+1
  double* rot = p.slotRot + (size_t)p.seed_id * 3 * p.max_a;
  for (int j = 0; j < a; ++j)
    for (int i = 0; i <= a; ++i) sh[i + j * sld] = (i <= j + 1) ? ch[i + j * cld] : 0.0;
  int lsq = 0, nrot = 0;
  factor_hessenberg(sh, sld, a, hn, R, rot, rot + 2 * p.max_a, &lsq, &nrot);
  SlotMeta mt;
  mt.a = a;
  mt.has_next = hn;
  mt.timestep = p.timestep;
  mt.N = N;
  mt.lsq = lsq;
  mt.nrot = nrot;
  mt.dense = mt.pad_ = 0;
  p.meta[p.seed_id] = mt;
}

template <int EPT, int NT>
__global__ void __launch_bounds__(NT) project_fp64_kernel(const ProjParams p) {
  constexpr int NWARPS = NT / 32;
  __shared__ double red[NWARPS * kMaxV];
  __shared__ double cvec[kMaxV];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int timestep = p.step ? *p.step : p.timestep;
  for (int t = blockIdx.x; t < p.nt; t += gridDim.x) {
    const SysDesc d = p.sys[t];
    const int N = d.H * d.W;
    const SlotMeta mt = p.meta[d.slot];
    if (mt.timestep != timestep || mt.N != N || mt.a == 0) continue;   // uniform per block
    const int a = mt.a;
    const int nv = mt.lsq ? a + 1 : a;
    const double* V = p.slotV + (size_t)d.slot * (p.max_a + 1) * p.ld;
    double r[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int pp = tid + k * NT;
      r[k] = (pp < N) ? d.b[pp] : 0.0;
    }
    // c = V^T r (c_i over the first nv basis vectors)
    const float* V32 = p.slotV32 ? p.slotV32 + (size_t)d.slot * (p.max_a + 1) * p.ld : nullptr;
    auto vget = [&](int i, int pp) -> double {
      return V32 ? (double)V32[(size_t)i * p.ld + pp] : V[(size_t)i * p.ld + pp];
    };
    block_partials<NT>(nv, [&](int i) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        const int pp = tid + k * NT;
        if (pp < N) s += vget(i, pp) * r[k];
      }
      return s;
    }, red);
    if (warp == 0) {
      for (int i = lane; i < nv; i += 32) cvec[i] = cross_warp<NT>(red, i);
      __syncwarp();
      const int sld = p.max_a + 1;
      const double* rot = p.slotRot + (size_t)d.slot * 3 * p.max_a;
      solve_projected_warp(cvec, a, mt.nrot, p.slotR + (size_t)d.slot * sld * p.max_a, sld, rot,
                           rot + 2 * p.max_a, lane);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
      const int pp = tid + k * NT;
      if (pp < N) {
        double xv = d.x[pp];
        for (int i = 0; i < a; ++i) xv = fma(cvec[i], vget(i, pp), xv);
        d.x[pp] = xv;
      }
    }
    __syncthreads();
  }
}

}  // namespace

__global__ void widen_kernel(const float* src, size_t src_ld, double* dst, size_t dst_ld, int n) {
  const int r = blockIdx.x;
  for (int q = threadIdx.x; q < n; q += blockDim.x) dst[(size_t)r * dst_ld + q] = (double)src[(size_t)r * src_ld + q];
}

__global__ void permute_kernel(double* dst, const double* src, const int* perm, int n, int gather) {
  const int q = blockIdx.x;
  const size_t from = gather ? (size_t)perm[q] : (size_t)q;
  const size_t to = gather ? (size_t)q : (size_t)perm[q];
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[to * n + i] = src[from * n + i];
}

cudaError_t launch_permute(double* dst, const double* src, const int* perm, int count, int n,
                           int gather, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  permute_kernel<<<count, 256, 0, st>>>(dst, src, perm, n, gather);
  return cudaGetLastError();
}

__global__ void to_bf16_kernel(__nv_bfloat16* dst, int ld, const double* src, int n, double scale) {
  const int q = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    dst[(size_t)q * ld + i] = __float2bfloat16_rn((float)(src[(size_t)q * n + i] * scale));
}

cudaError_t launch_to_bf16(__nv_bfloat16* dst, int ld, const double* src, int count, int n,
                           double scale, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  to_bf16_kernel<<<count, 256, 0, st>>>(dst, ld, src, n, scale);
  return cudaGetLastError();
}

cudaError_t launch_widen(const float* src, size_t src_ld, double* dst, size_t dst_ld, int n, int rows,
                         cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  widen_kernel<<<rows, 256, 0, st>>>(src, src_ld, dst, dst_ld, n);
  return cudaGetLastError();
}

cudaError_t launch_factor(const FactorParams& p, cudaStream_t st) {
  factor_kernel<<<p.count > 0 ? p.count : 1, 256, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_project_fp64(const ProjParams& p, int ept, int nt, cudaStream_t st) {
  if (ept == 4 && nt == 256) project_fp64_kernel<4, 256><<<p.nt, 256, 0, st>>>(p);
  else if (ept == 8 && nt == 128) project_fp64_kernel<8, 128><<<p.nt, 128, 0, st>>>(p);
  else if (ept == 8 && nt == 512) project_fp64_kernel<8, 512><<<p.nt, 512, 0, st>>>(p);
  else if (ept == 16 && nt == 1024) project_fp64_kernel<16, 1024><<<p.nt, 1024, 0, st>>>(p);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace kp
