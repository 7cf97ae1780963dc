// kp_proj_tc.cu -- the projection contraction of Sec. 3, Phase 2,
//     C[t][i] = sum_k B[t][k] V[i][k]     (c_t = V_a^T b_t for every target t)
// on the 5th-generation tensor cores: BF16 inputs, FP32 accumulation in TMEM.
//
// One CTA computes a 128-target x 48-vector tile of C over the whole K (the
// grid size N = H*W): TMA streams 128x64 target and 48x64 basis tiles (128-byte
// swizzle) through a 4-stage shared-memory ring, one elected thread issues
// tcgen05.mma (M=128, N=48, K=16) into a TMEM accumulator, and all four warps
// read their 32 TMEM lanes back with tcgen05.ld for the epilogue.  Every
// mbarrier wait is bounded: on timeout the CTA records an error, waits (bounded)
// for its copies in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include "kp_internal.cuh"

namespace kp {
namespace {

constexpr int kTileM = 128;         // targets per tile (TMEM lanes)
constexpr int kTileN = 48;          // basis vectors per tile (>= a + 1 for a <= 47)
constexpr int kTileK = 64;          // BF16 elements per 128-byte swizzle row
constexpr int kStages = 4;
constexpr uint32_t kBytesA = kTileM * kTileK * 2;
constexpr uint32_t kBytesB = kTileN * kTileK * 2;
constexpr uint32_t kTmemCols = 64;
constexpr long long kSpinLimit = 1ll << 26;   // ~seconds of polling, far above any tile

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long long i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor: K-major tile with 128-byte swizzle,
// 8-row core-matrix groups 1024 bytes apart (SBO), sm_100 descriptor version.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                   // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset
  d |= (uint64_t)1 << 46;                   // descriptor version
  d |= (uint64_t)2 << 61;                   // SWIZZLE_128B
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4)                          // D format F32
         | (1u << 7)                        // A format BF16
         | (1u << 10)                       // B format BF16
         | ((uint32_t)(N >> 3) << 17)       // N / 8
         | ((uint32_t)(M >> 4) << 24);      // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
      " [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct __align__(1024) TcSmem {
  __nv_bfloat16 A[kStages][kTileM * kTileK];   // target tiles, 16 KB each
  __nv_bfloat16 B[kStages][kTileN * kTileK];   // basis tiles, 6 KB each (1024-aligned: 6144)
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t done;
  uint32_t tmem_base;
  int abort;
};

__global__ void __launch_bounds__(128, 1)
proj_gemm_bf16_kernel(const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapV,
                      const ProjTile* tiles, int ntiles, int K, float* C, int ldc, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw_tc[];
  // align the dynamic window to 1024 bytes (128-byte swizzle atoms)
  TcSmem& sm = *reinterpret_cast<TcSmem*>(
      (reinterpret_cast<uintptr_t>(smem_raw_tc) + 1023) & ~(uintptr_t)1023);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nk = (K + kTileK - 1) / kTileK;
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&sm.full[s], 1);
      mbar_init(&sm.empty[s], 1);
    }
    mbar_init(&sm.done, 1);
    sm.abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&sm.tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sm.tmem_base;
  constexpr uint32_t idesc = idesc_bf16_f32(kTileM, kTileN);
  uint32_t issued = 0;                            // TMA stage loads issued (producer thread)
  uint32_t base_phase = 0;                        // K chunks of earlier tiles of this CTA

  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const ProjTile tile = tiles[t];
    const int round = (t - (int)blockIdx.x) / (int)gridDim.x;   // tiles already done by this CTA
    const int kc0 = tile.kc1 > 0 ? tile.kc0 : 0;
    const int nkt = tile.kc1 > 0 ? tile.kc1 - tile.kc0 : nk;
    if (warp == 0 && lane == 0) {
      // TMA producer
      for (int kc = 0; kc < nkt; ++kc) {
        const uint32_t it = base_phase + kc;
        const int s = it % kStages;
        const uint32_t use = it / kStages;
        if (use > 0 && !mbar_wait(&sm.empty[s], (use - 1) & 1)) { sm.abort = 1; break; }
        mbar_expect_tx(&sm.full[s], kBytesA + kBytesB);
        tma_load_2d(sm.A[s], &mapB, (kc0 + kc) * kTileK, tile.row0, &sm.full[s]);
        tma_load_2d(sm.B[s], &mapV, (kc0 + kc) * kTileK, tile.vrow0, &sm.full[s]);
        issued = it + 1;
      }
    } else if (warp == 1 && lane == 0) {
      // MMA issuer
      for (int kc = 0; kc < nkt; ++kc) {
        const uint32_t it = base_phase + kc;
        const int s = it % kStages;
        const uint32_t use = it / kStages;
        if (!mbar_wait(&sm.full[s], use & 1)) { sm.abort = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint64_t ad = smem_desc_sw128(smem_u32(sm.A[s]));
        const uint64_t bd = smem_desc_sw128(smem_u32(sm.B[s]));
#pragma unroll
        for (int kk = 0; kk < kTileK / 16; ++kk)     // 16 BF16 = 32 bytes per MMA
          mma_bf16(tmem, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc,
                   (kc > 0 || kk > 0) ? 1u : 0u);
        mma_commit(&sm.empty[s]);                  // frees the stage when the MMAs finish
      }
      mma_commit(&sm.done);
    }
    __syncwarp();
    // epilogue: all four warps, each over its 32 TMEM lanes (= targets)
    const bool ok = mbar_wait(&sm.done, (uint32_t)(round & 1));
    __syncthreads();
    if (!ok || sm.abort) {
      if (tid == 0) atomicExch(err, 1);
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int r = warp * 32 + lane;
#pragma unroll
    for (int c0 = 0; c0 < kTileN; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      if (r < tile.count) {
        float* crow = C + (size_t)(tile.crow0 + r) * ldc + tile.ccol0 + c0;
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (c0 + i < tile.nv) {
            if (tile.atomic) atomicAdd(crow + i, v[i]);
            else crow[i] = v[i];
          }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    base_phase += (uint32_t)nkt;
  }
  __syncthreads();
  if (sm.abort && warp == 0 && lane == 0) {
    // let the copies this CTA issued land before its shared memory goes away:
    // the last load on stage s completes phase (its use index) & 1
    for (int s = 0; s < kStages; ++s) {
      if (issued == 0) break;
      const uint32_t last = issued - 1;
      const uint32_t back = (last % kStages + kStages - (uint32_t)s) % kStages;
      if (back > last) continue;                  // stage s never loaded
      (void)mbar_wait(&sm.full[s], ((last - back) / kStages) & 1);
    }
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
}

}  // namespace

size_t proj_gemm_smem_bytes() { return sizeof(TcSmem) + 1024; }

cudaError_t make_bf16_map(void* map, const void* base, int rows, int cols, int ld, int box_rows) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kTileK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                      const_cast<void*>(base), dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_proj_gemm_bf16(const CUtensorMap& mapB, const CUtensorMap& mapV,
                                  const ProjTile* tiles, int ntiles, int K, float* C, int ldc,
                                  int* err, int grid, cudaStream_t st) {
  if (ntiles <= 0) return cudaSuccess;
  const size_t smem = proj_gemm_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(proj_gemm_bf16_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  proj_gemm_bf16_kernel<<<grid, 128, smem, st>>>(mapB, mapV, tiles, ntiles, K, C, ldc, err);
  return cudaGetLastError();
}

}  // namespace kp
