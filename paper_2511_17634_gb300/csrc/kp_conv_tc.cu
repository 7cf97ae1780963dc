// kp_conv_tc.cu -- 3x3 convolutions of the learned-initial-guess network as
// implicit GEMMs on the tcgen05 tensor cores, with no im2col matrix in memory.
//
// Activations live in a padded-column BF16 layout: per sample and per group of
// 8 channels ("chunk") a plane of rows of 16 bytes (8 channels), row
// halo + i*(H+2) + 1 + j holding pixel (i, j) and zero rows around every
// column (j = -1, j = H) and around the whole image (halo = H + 3 rows at each
// end).  In that layout the 3x3 tap (di, dj) of output row r is input row
// r + di*(H+2) + dj, and the zero rows supply the zero padding, so the A
// operand of tap t is the staged input tile itself shifted by a whole number
// of 16-byte rows.  With the no-swizzle K-major operand layout (8-row x
// 16-byte core matrices, SBO = 128 bytes between row groups, LBO = one chunk
// plane between K halves) a row shift is a plain change of the descriptor's
// start address.
//
//   Z[r][co] = bias[co] + sum_t sum_c X[r + off(t)][c] W[co][c][t]
//
// One CTA (persistent) processes super tiles of 8 x 128 padded rows: a
// producer thread stages the input rows of a super tile plus halos with bulk
// copies (cp.async.bulk, two stages), one thread issues 9 taps x (C_in / 16)
// MMAs (M = 128 rows, N = 16 or 32 output channels, K = 16) per 128-row tile
// into a double-buffered TMEM accumulator, and four warps read TMEM back
// (tcgen05.ld), add the bias, apply ReLU and store BF16 rows (or FP32 planes
// for the last layer).  Every mbarrier wait is bounded; on timeout the CTA
// records an error and leaves after its copies and MMAs have landed.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "kp_internal.cuh"

namespace kp {
namespace {

constexpr int kMT = 8;                  // 128-row tiles per super tile (input window re-read
                                        // factor (1024 + 2 halo) / 1024 = 1.26 at 128x128)
constexpr int kConvThreads = 192;       // warps 0-3 epilogue, 4 producer, 5 MMA issuer
constexpr long long kConvSpin = 1ll << 26;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void bar_init(uint64_t* b, uint32_t n) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(n) : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait that also gives up when another role has aborted.
__device__ __forceinline__ bool bar_wait(uint64_t* b, uint32_t parity, const volatile int* abort) {
  for (long long i = 0; i < kConvSpin; ++i) {
    if (bar_try(b, parity)) return true;
    if ((i & 255) == 255 && *abort) return false;
  }
  return false;
}

__device__ __forceinline__ void bar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}

__device__ __forceinline__ void bar_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}

// contiguous global -> shared copy (16-byte aligned, multiple of 16 bytes)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          su32(dst)),
      "l"(src), "r"(bytes), "r"(su32(b))
      : "memory");
}

// K-major operand without swizzle: core matrices of 8 rows x 16 bytes, rows
// 16 bytes apart; lbo = bytes between the two K halves of an MMA (one chunk
// plane), sbo = bytes between 8-row groups.
__device__ __forceinline__ uint64_t desc_plain(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;                    // descriptor version (sm_100 family)
  return d;                                  // swizzle mode 0: none
}

__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// (no memory clobber: the MMA reads shared memory through the async proxy,
// and volatile asm keeps it ordered after the barrier waits and fences and
// before the commit that publishes its completion)
__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit_to(uint64_t* b) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(b))
               : "memory");
}

__device__ __forceinline__ void tmem_ld_x16(uint32_t taddr, float (&v)[16]) {
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

// zeros to 16 TMEM columns of the warp's 32 lanes (the caller waits with
// tcgen05.wait::st before the columns are handed to the MMAs)
__device__ __forceinline__ void tmem_zero_x16(uint32_t taddr) {
  const uint32_t z = 0u;
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};" ::"r"(taddr),
      "r"(z)
      : "memory");
}

struct ConvArgs {
  const __nv_bfloat16* in;     // [B][CIC][Rp][8]
  const __nv_bfloat16* wf;     // [9][CIC][NOUT][8]
  const float* bias;           // [cout]
  __nv_bfloat16* out_pad;      // [B][4][Rp][8] (hidden layers)
  float* out_f32;              // [B][cout][H*W] (last layer)
  int B, H, W, halo, Rp, nst, cout;
  int* err;
};

// Shared memory: two input stages of CIC chunk planes of L rows, the weights,
// then the barriers.
template <int CIC, int NOUT>
struct ConvLayout {
  static __host__ __device__ uint32_t L(int halo) { return (uint32_t)(kMT * 128 + 2 * halo); }
  static __host__ __device__ uint32_t stage_bytes(int halo) { return CIC * L(halo) * 16u; }
  static __host__ __device__ uint32_t w_bytes() { return 9u * CIC * NOUT * 16u; }
  static __host__ __device__ uint32_t bar_off(int halo) { return 2 * stage_bytes(halo) + w_bytes(); }
  static __host__ __device__ size_t total(int halo) { return bar_off(halo) + 128 + 128; }
};

template <int CIC, int NOUT, bool F32OUT>
__global__ void __launch_bounds__(kConvThreads, 1) conv3x3_tc_kernel(const ConvArgs a) {
  static_assert(F32OUT || NOUT == 32 || NOUT == 16, "hidden layers write NOUT / 8 chunks of 8 channels");
  using Lay = ConvLayout<CIC, NOUT>;
  extern __shared__ __align__(128) unsigned char cs[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(cs) + 127) & ~(uintptr_t)127);
  const uint32_t L = Lay::L(a.halo);
  const uint32_t SB = Lay::stage_bytes(a.halo);
  unsigned char* stage0 = base;
  unsigned char* wsm = base + 2 * SB;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + Lay::bar_off(a.halo));
  uint64_t* full = bars;          // [2] input stage landed
  uint64_t* mdone = bars + 2;     // [2] MMAs of a super tile done (stage and TMEM buffer)
  uint64_t* tempty = bars + 4;    // [2] epilogue finished reading a TMEM buffer
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 6);
  volatile int* abort = reinterpret_cast<volatile int*>(bars + 7);
  constexpr uint32_t kCols = 2 * kMT * NOUT;   // 512 or 256 TMEM columns
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int total = a.B * a.nst;

  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      bar_init(&full[s], 1);
      bar_init(&mdone[s], 1);
      bar_init(&tempty[s], 4);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // weights -> shared memory (read by the tensor cores: async proxy)
  {
    const uint4* src = reinterpret_cast<const uint4*>(a.wf);
    uint4* dst = reinterpret_cast<uint4*>(wsm);
    for (uint32_t q = tid; q < Lay::w_bytes() / 16; q += kConvThreads) dst[q] = src[q];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int HP = a.H + 2;

  if (warp == 4) {
    if (lane == 0) {
      // producer: input rows [q0, q0 + L) of every chunk plane (plane row =
      // halo + padded row, so the window starts at plane row q0)
      uint32_t issued = 0;
      int it = 0;
      for (int st = blockIdx.x; st < total; st += gridDim.x, ++it) {
        const int s = it & 1;
        const uint32_t u = (uint32_t)it >> 1;
        if (u > 0 && !bar_wait(&mdone[s], (u - 1) & 1, abort)) { *abort = 1; break; }
        const int b = st / a.nst;
        const size_t q0 = (size_t)(st - b * a.nst) * kMT * 128;
        bar_expect(&full[s], SB);
        for (int c = 0; c < CIC; ++c)
          bulk_g2s(stage0 + s * SB + (size_t)c * L * 16, a.in + (((size_t)b * CIC + c) * a.Rp + q0) * 8, L * 16,
                   &full[s]);
        issued = (uint32_t)it + 1;
      }
      if (*abort) {
        // let the last copies of each stage land before the shared memory is released
        volatile int never = 0;
        for (uint32_t k = issued > 2 ? issued - 2 : 0; k < issued; ++k)
          (void)bar_wait(&full[k & 1], (k >> 1) & 1, &never);
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_f16(128, NOUT);
      uint32_t committed = 0;
      int it = 0;
      for (int st = blockIdx.x; st < total; st += gridDim.x, ++it) {
        const int s = it & 1;
        const uint32_t u = (uint32_t)it >> 1;
        if (!bar_wait(&full[s], u & 1, abort)) { *abort = 1; break; }
        if (u > 0 && !bar_wait(&tempty[s], (u - 1) & 1, abort)) { *abort = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t sa = su32(stage0 + s * SB);
        const uint32_t sw = su32(wsm);
#pragma unroll 1
        for (int q = 0; q < kMT; ++q) {
          const uint32_t d = tmem + (uint32_t)(s * kMT * NOUT + q * NOUT);
#pragma unroll
          for (int t = 0; t < 9; ++t) {
            const int row = a.halo + q * 128 + (t / 3 - 1) * HP + (t % 3 - 1);
#pragma unroll
            for (int kc = 0; kc < CIC / 2; ++kc) {
              const uint64_t ad = desc_plain(sa + (uint32_t)(2 * kc) * L * 16 + (uint32_t)row * 16, L * 16, 128);
              const uint64_t bd = desc_plain(sw + (uint32_t)((t * CIC + 2 * kc) * NOUT * 16), NOUT * 16, 128);
              mma_f16(d, ad, bd, idesc, (t > 0 || kc > 0) ? 1u : 0u);
            }
          }
        }
        mma_commit_to(&mdone[s]);
        committed = (uint32_t)it + 1;
      }
      if (*abort && committed > 0) {
        // the TMEM may only be released once the issued MMAs have finished
        const uint32_t k = committed - 1;
        volatile int never = 0;
        (void)bar_wait(&mdone[k & 1], (k >> 1) & 1, &never);
      }
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32w..32w+31 = rows of each 128-row tile
    int it = 0;
    for (int st = blockIdx.x; st < total; st += gridDim.x, ++it) {
      const int s = it & 1;
      const uint32_t u = (uint32_t)it >> 1;
      if (!bar_wait(&mdone[s], u & 1, abort)) { *abort = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int b = st / a.nst;
      const int q0 = (st - b * a.nst) * kMT * 128;
#pragma unroll 1
      for (int q = 0; q < kMT; ++q) {
        const int R = q0 + q * 128 + warp * 32 + lane;        // padded row
        const int i = R / HP;
        const int jj = R - i * HP - 1;
        const bool valid = i < a.W && jj >= 0 && jj < a.H;
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(s * kMT * NOUT + q * NOUT);
        float v[NOUT];
#pragma unroll
        for (int c0 = 0; c0 < NOUT; c0 += 16) {
          float w16[16];
          tmem_ld_x16(taddr + (uint32_t)c0, w16);
#pragma unroll
          for (int k = 0; k < 16; ++k) v[c0 + k] = w16[k];
        }
        if (F32OUT) {
          if (valid) {
#pragma unroll
            for (int co = 0; co < NOUT; ++co)
              if (co < a.cout)
                a.out_f32[((size_t)b * a.cout + co) * a.H * a.W + (size_t)i * a.H + jj] = v[co] + a.bias[co];
          }
        } else {
#pragma unroll
          for (int cc = 0; cc < NOUT / 8; ++cc) {
            uint32_t pk[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int c0 = cc * 8 + 2 * e;
              float x0 = 0.f, x1 = 0.f;
              if (valid && c0 < a.cout) x0 = fmaxf(v[c0] + a.bias[c0], 0.f);
              if (valid && c0 + 1 < a.cout) x1 = fmaxf(v[c0 + 1] + a.bias[c0 + 1], 0.f);
              __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
              pk[e] = *reinterpret_cast<uint32_t*>(&h2);
            }
            uint4* dst = reinterpret_cast<uint4*>(a.out_pad + (((size_t)b * (NOUT / 8) + cc) * a.Rp + a.halo + R) * 8);
            *dst = make_uint4(pk[0], pk[1], pk[2], pk[3]);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) bar_arrive(&tempty[s]);
    }
  }
  __syncthreads();
  if (tid == 0 && *abort) atomicOr(a.err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
  }
}

// ---------------------------------------------------------------------------
// Column-aligned variant for 64 < H <= 128: one 128-row tile is the pixel
// rows j = 0..127 of one image column, so the column shift di of tap (di, dj)
// moves a whole tile.  The A tile of input column s shifted by dj then feeds
// all three column taps at once: with B = [W(-1,dj); W(0,dj); W(+1,dj)]
// (N = 3 x NOUT), the three NOUT-wide groups of the product belong to output
// columns s+1, s, s-1, and with the output accumulators laid out in
// descending column order in TMEM (output column o at NOUT (K-1-(o-i0))) those
// three are adjacent: one MMA of N = 3 NOUT accumulates into all of them.
// Per output column and K step that is 3 MMAs of N = 3 NOUT reading three A
// tiles instead of 9 MMAs of N = NOUT reading nine, so the shared-memory
// operand traffic per useful multiply-add falls by about 2x.
//
// A super tile is kCT output columns [i0, i0 + Kv) of one sample; its input
// window is columns i0-1 .. i0+Kv (whole padded columns, zero rows included).
// Every MMA accumulates: the accumulators are zeroed once after allocation and
// each epilogue stores zeros over the columns it has read, so no input column
// needs a separate MMA for the output columns it reaches first.  Rows j >= H
// of a tile (H < 128) read the next column or the slack rows at the end of
// the stage and land in discarded D rows.
constexpr int kCT = 8;                  // output columns per super tile
constexpr int kColEpiWarps = 8;         // two epilogue warps per TMEM lane quadrant
constexpr int kColThreads = 32 * (kColEpiWarps + 2);   // + producer warp + MMA warp

template <int CIC, int NOUT>
struct ColLayout {
  static __host__ __device__ uint32_t L(int H) {
    return (uint32_t)((kCT + 2) * (H + 2) + (H < 128 ? 128 - H : 0));
  }
  // input stages: four of the two-chunk windows (41.6 KB at 128x128), two of
  // the four-chunk ones; the TMEM accumulator is double-buffered either way
  static constexpr int NS = CIC == 2 ? 4 : 2;
  static __host__ __device__ uint32_t stage_bytes(int H) { return CIC * L(H) * 16u; }
  static __host__ __device__ uint32_t w_bytes() { return 9u * CIC * NOUT * 16u; }
  static __host__ __device__ uint32_t bar_off(int H) { return NS * stage_bytes(H) + w_bytes(); }
  static __host__ __device__ size_t total(int H) { return bar_off(H) + 128 + 128; }
};

template <int CIC, int NOUT, bool F32OUT>
__global__ void __launch_bounds__(kColThreads, 1) conv3x3_col_kernel(const ConvArgs a) {
  static_assert(F32OUT || NOUT == 32 || NOUT == 16, "hidden layers write NOUT / 8 chunks of 8 channels");
  using Lay = ColLayout<CIC, NOUT>;
  extern __shared__ __align__(128) unsigned char cs[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(cs) + 127) & ~(uintptr_t)127);
  const uint32_t L = Lay::L(a.H);
  const uint32_t SB = Lay::stage_bytes(a.H);
  unsigned char* stage0 = base;
  constexpr int NS = Lay::NS;
  unsigned char* wsm = base + NS * SB;
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + Lay::bar_off(a.H));
  uint64_t* full = bars;          // [NS] input stage landed
  uint64_t* sfree = bars + NS;    // [NS] MMAs reading an input stage done
  uint64_t* tfull = bars + 2 * NS;      // [2] MMAs of a super tile done (TMEM buffer ready)
  uint64_t* tempty = bars + 2 * NS + 2; // [2] epilogue finished reading a TMEM buffer
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * NS + 4);
  volatile int* abort = reinterpret_cast<volatile int*>(bars + 2 * NS + 5);
  constexpr uint32_t kCols = 2 * kCT * NOUT;   // 512 or 256 TMEM columns
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int HP = a.H + 2;
  const int nct = (a.W + kCT - 1) / kCT;
  const int total = a.B * nct;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      bar_init(&full[s], 1);
      bar_init(&sfree[s], 1);
    }
    for (int t = 0; t < 2; ++t) {
      bar_init(&tfull[t], 1);
      bar_init(&tempty[t], kColEpiWarps);
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // weights -> shared memory as [dj][chunk][(di + 1) NOUT + co][8] from the
  // tap-major global layout [t = 3 (di + 1) + dj + 1][chunk][co][8]
  {
    const uint4* src = reinterpret_cast<const uint4*>(a.wf);
    uint4* dst = reinterpret_cast<uint4*>(wsm);
    for (uint32_t q = tid; q < Lay::w_bytes() / 16; q += kColThreads) {
      const uint32_t co = q % NOUT, c8 = (q / NOUT) % CIC, t = q / (NOUT * CIC);
      dst[((t % 3) * CIC + c8) * 3 * NOUT + (t / 3) * NOUT + co] = src[q];
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  // the accumulators start at zero and every epilogue returns the columns it
  // read to zero, so every MMA accumulates (no first-touch MMA of its own)
  if (warp < kColEpiWarps) {
    const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;
    for (uint32_t col = (uint32_t)(warp >> 2) * 16; col < 2u * kCT * NOUT; col += (kColEpiWarps / 4) * 16)
      tmem_zero_x16(tmem + lanes + col);
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (warp == kColEpiWarps) {
    if (lane == 0) {
      // producer: plane rows of input columns i0-1 .. i0+Kv of every chunk
      // plane (column i starts at plane row halo + i HP; column -1 is the
      // zero halo, and column W lies inside the zero tail)
      uint32_t issued = 0;
      int it = 0;
      for (int st = blockIdx.x; st < total; st += gridDim.x, ++it) {
        const int s = it % NS;
        const uint32_t u = (uint32_t)(it / NS);
        if (u > 0 && !bar_wait(&sfree[s], (u - 1) & 1, abort)) { *abort = 1; break; }
        const int b = st / nct;
        const int i0 = (st - b * nct) * kCT;
        const int kv = min(kCT, a.W - i0);
        const size_t q0 = (size_t)(a.halo + (i0 - 1) * HP);
        const uint32_t rows = (uint32_t)(kv + 2) * HP;
        bar_expect(&full[s], CIC * rows * 16);
        for (int c = 0; c < CIC; ++c)
          bulk_g2s(stage0 + s * SB + (size_t)c * L * 16, a.in + (((size_t)b * CIC + c) * a.Rp + q0) * 8, rows * 16,
                   &full[s]);
        issued = (uint32_t)it + 1;
      }
      if (*abort) {
        volatile int never = 0;
        for (uint32_t k = issued > (uint32_t)NS ? issued - NS : 0; k < issued; ++k)
          (void)bar_wait(&full[k % NS], (k / NS) & 1, &never);
      }
    }
  } else if (warp == kColEpiWarps + 1) {
    if (lane == 0) {
      uint32_t committed = 0;
      int it = 0;
      for (int st = blockIdx.x; st < total; st += gridDim.x, ++it) {
        const int s = it % NS, tb = it & 1;
        const uint32_t u = (uint32_t)(it / NS), ut = (uint32_t)it >> 1;
        if (!bar_wait(&full[s], u & 1, abort)) { *abort = 1; break; }
        if (ut > 0 && !bar_wait(&tempty[tb], (ut - 1) & 1, abort)) { *abort = 1; break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int b = st / nct;
        const int i0 = (st - b * nct) * kCT;
        const int kv = min(kCT, a.W - i0);
        // descriptors: only the start-address field (bits 0..13, the address
        // in 16-byte units) differs between the MMAs of a tile, and it never
        // carries out of its 14 bits (shared-memory addresses are below
        // 256 KB), so each MMA's descriptors are the tile's base descriptors
        // plus an offset in 16-byte rows
        const uint64_t abase = desc_plain(su32(stage0 + s * SB), L * 16, 128);
        const uint64_t bbase = desc_plain(su32(wsm), 3 * NOUT * 16, 128);
        const uint32_t dbase = tmem + (uint32_t)(tb * kCT * NOUT);
        const int cb = max(i0 - 1, 0), ce = min(i0 + kv, a.W - 1);   // input columns inside the image
#pragma unroll 1
        for (int c = cb; c <= ce; ++c) {
          // groups g = di + 1 in [g0, g1] reach output columns c + 1 - g
          // inside the tile
          const int g0 = max(0, c + 2 - i0 - kv), g1 = min(2, c + 1 - i0);
          const uint32_t idesc = idesc_f16(128, (g1 - g0 + 1) * NOUT);
          // A rows of input column c shifted by dj - 1: (c - i0 + 1) HP + dj
          const uint64_t acol = abase + (uint64_t)((c - i0 + 1) * HP);
          // accumulators of output columns c + 1 - g0 .. c + 1 - g1 (descending
          // order in TMEM), starting at output column c + 1 - g0
          const uint32_t d = dbase + (uint32_t)(NOUT * (kCT - 2 - c + i0 + g0));
#pragma unroll
          for (int dj = 0; dj < 3; ++dj) {
#pragma unroll
            for (int kc = 0; kc < CIC / 2; ++kc) {
              const uint64_t ad = acol + (uint64_t)(2 * kc * L + dj);
              const uint64_t bd = bbase + (uint64_t)((dj * CIC + 2 * kc) * 3 * NOUT + g0 * NOUT);
              mma_f16(d, ad, bd, idesc, 1u);
            }
          }
        }
        mma_commit_to(&sfree[s]);                   // the input stage may be refilled
        mma_commit_to(&tfull[tb]);                  // the accumulators are ready
        committed = (uint32_t)it + 1;
      }
      if (*abort && committed > 0) {
        const uint32_t k = committed - 1;
        volatile int never = 0;
        (void)bar_wait(&tfull[k & 1], (k >> 1) & 1, &never);
      }
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = pixel rows j of
    // every (kColEpiWarps / 4)-th output column, starting at column w / 4
    int it = 0;
    for (int st = blockIdx.x; st < total; st += gridDim.x, ++it) {
      const int tb = it & 1;
      const uint32_t ut = (uint32_t)it >> 1;
      if (!bar_wait(&tfull[tb], ut & 1, abort)) { *abort = 1; break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int b = st / nct;
      const int i0 = (st - b * nct) * kCT;
      const int kv = min(kCT, a.W - i0);
      const int quad = warp & 3;
      const int j = quad * 32 + lane;
      const bool valid_j = j < a.H;
#pragma unroll 1
      for (int q = warp >> 2; q < kv; q += kColEpiWarps / 4) {
        const int o = i0 + q;
        const uint32_t taddr =
            tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(tb * kCT * NOUT + NOUT * (kCT - 1 - q));
        float v[NOUT];
#pragma unroll
        for (int c0 = 0; c0 < NOUT; c0 += 16) {
          float w16[16];
          tmem_ld_x16(taddr + (uint32_t)c0, w16);
#pragma unroll
          for (int k = 0; k < 16; ++k) v[c0 + k] = w16[k];
        }
        if (!valid_j) continue;
        if (F32OUT) {
#pragma unroll
          for (int co = 0; co < NOUT; ++co)
            if (co < a.cout)
              a.out_f32[((size_t)b * a.cout + co) * a.H * a.W + (size_t)o * a.H + j] = v[co] + a.bias[co];
        } else {
          const size_t prow = (size_t)a.halo + (size_t)o * HP + 1 + j;
#pragma unroll
          for (int cc = 0; cc < NOUT / 8; ++cc) {
            uint32_t pk[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int c0 = cc * 8 + 2 * e;
              const float x0 = c0 < a.cout ? fmaxf(v[c0] + a.bias[c0], 0.f) : 0.f;
              const float x1 = c0 + 1 < a.cout ? fmaxf(v[c0 + 1] + a.bias[c0 + 1], 0.f) : 0.f;
              __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
              pk[e] = *reinterpret_cast<uint32_t*>(&h2);
            }
            *reinterpret_cast<uint4*>(a.out_pad + (((size_t)b * (NOUT / 8) + cc) * a.Rp + prow) * 8) =
                make_uint4(pk[0], pk[1], pk[2], pk[3]);
          }
        }
      }
      // return the columns this warp read to zero for the MMAs of tile it + 2
#pragma unroll 1
      for (int q = warp >> 2; q < kv; q += kColEpiWarps / 4) {
        const uint32_t taddr =
            tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(tb * kCT * NOUT + NOUT * (kCT - 1 - q));
#pragma unroll
        for (int c0 = 0; c0 < NOUT; c0 += 16) tmem_zero_x16(taddr + (uint32_t)c0);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) bar_arrive(&tempty[tb]);
    }
  }
  __syncthreads();
  if (tid == 0 && *abort) atomicOr(a.err, 1);
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
  }
}

// Wf[t][c8][co][e] = W[co][c8*8+e][t] (0 outside C_in x C_out)
__global__ void conv_weights_kernel(const float* Wl, int cin, int cout, int cic, int nout, __nv_bfloat16* wf) {
  const int n = 9 * cic * nout * 8;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const int e = q & 7;
    const int co = (q >> 3) % nout;
    const int c8 = (q >> 3) / nout % cic;
    const int t = (q >> 3) / nout / cic;
    const int c = c8 * 8 + e;
    const float v = (c < cin && co < cout) ? Wl[((size_t)co * cin + c) * 9 + t] : 0.f;
    wf[q] = __float2bfloat16_rn(v);
  }
}

// FP32 planes [B][C][H*W] -> padded rows [B][chunks][Rp][8] (pixel rows only;
// the zero rows are never written)
__global__ void planes_to_padded_kernel(const float* X, int C, int chunks, int H, int W, int halo, int Rp,
                                        __nv_bfloat16* out) {
  const int b = blockIdx.y;
  const int P = H * W;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const int i = p / H, j = p - i * H;
    const size_t row = (size_t)halo + (size_t)i * (H + 2) + 1 + j;
    for (int c8 = 0; c8 < chunks; ++c8) {
      uint32_t pk[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int c = c8 * 8 + 2 * e;
        const float x0 = c < C ? X[((size_t)b * C + c) * P + p] : 0.f;
        const float x1 = c + 1 < C ? X[((size_t)b * C + c + 1) * P + p] : 0.f;
        __nv_bfloat162 h2 = __floats2bfloat162_rn(x0, x1);
        pk[e] = *reinterpret_cast<uint32_t*>(&h2);
      }
      *reinterpret_cast<uint4*>(out + (((size_t)b * chunks + c8) * Rp + row) * 8) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
  }
}

template <int CIC, int NOUT, bool F32OUT>
cudaError_t launch_conv_t(const ConvArgs& a, int sms, cudaStream_t st) {
  auto k = conv3x3_tc_kernel<CIC, NOUT, F32OUT>;
  const size_t smem = ConvLayout<CIC, NOUT>::total(a.halo);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int total = a.B * a.nst;
  k<<<std::min(total, sms), kConvThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int CIC, int NOUT, bool F32OUT>
cudaError_t launch_col_t(const ConvArgs& a, int sms, cudaStream_t st) {
  auto k = conv3x3_col_kernel<CIC, NOUT, F32OUT>;
  const size_t smem = ColLayout<CIC, NOUT>::total(a.H);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int total = a.B * ((a.W + kCT - 1) / kCT);
  k<<<std::min(total, sms), kColThreads, smem, st>>>(a);
  return cudaGetLastError();
}

// the column-aligned kernel needs a whole column in one 128-row tile and wastes
// the rows past H, so it serves 64 < H <= 128
bool use_col(const ConvGeom& g) { return g.H > 64 && g.H <= 128; }

}  // namespace

ConvGeom conv_geom(int H, int W) {
  ConvGeom g;
  g.H = H;
  g.W = W;
  g.halo = H + 3;
  const int rows = W * (H + 2);
  const int ntile = (rows + 127) / 128;
  g.nst = (ntile + kMT - 1) / kMT;
  g.Rp = 2 * g.halo + g.nst * kMT * 128;
  return g;
}

size_t conv_smem_bytes(const ConvGeom& g, int cic, int nout) {
  if (use_col(g)) {
    if (cic == 2 && nout == 32) return ColLayout<2, 32>::total(g.H);
    if (cic == 4 && nout == 32) return ColLayout<4, 32>::total(g.H);
    if (cic == 4 && nout == 16) return ColLayout<4, 16>::total(g.H);
    if (cic == 2 && nout == 16) return ColLayout<2, 16>::total(g.H);
    return 0;
  }
  if (cic == 2 && nout == 32) return ConvLayout<2, 32>::total(g.halo);
  if (cic == 4 && nout == 32) return ConvLayout<4, 32>::total(g.halo);
  if (cic == 4 && nout == 16) return ConvLayout<4, 16>::total(g.halo);
  if (cic == 2 && nout == 16) return ConvLayout<2, 16>::total(g.halo);
  return 0;
}

cudaError_t launch_conv_weights(const float* Wl, int cin, int cout, int cic, int nout, __nv_bfloat16* wf,
                                cudaStream_t st) {
  const int n = 9 * cic * nout * 8;
  conv_weights_kernel<<<(n + 255) / 256, 256, 0, st>>>(Wl, cin, cout, cic, nout, wf);
  return cudaGetLastError();
}

cudaError_t launch_planes_to_padded(const float* X, int B, int C, int chunks, const ConvGeom& g,
                                    __nv_bfloat16* out, cudaStream_t st) {
  const int P = g.H * g.W;
  planes_to_padded_kernel<<<dim3(std::min((P + 255) / 256, 1024), B), 256, 0, st>>>(X, C, chunks, g.H, g.W,
                                                                                   g.halo, g.Rp, out);
  return cudaGetLastError();
}

cudaError_t launch_conv3x3(const __nv_bfloat16* in, int B, int cic, const __nv_bfloat16* wf, const float* bias,
                           int cout, int nout, const ConvGeom& g, __nv_bfloat16* out_pad, float* out_f32,
                           int* err, int sms, cudaStream_t st) {
  ConvArgs a;
  a.in = in; a.wf = wf; a.bias = bias; a.out_pad = out_pad; a.out_f32 = out_f32;
  a.B = B; a.H = g.H; a.W = g.W; a.halo = g.halo; a.Rp = g.Rp; a.nst = g.nst; a.cout = cout; a.err = err;
  if (use_col(g)) {
    if (!out_f32 && cic == 2 && nout == 32) return launch_col_t<2, 32, false>(a, sms, st);
    if (!out_f32 && cic == 4 && nout == 32) return launch_col_t<4, 32, false>(a, sms, st);
    if (!out_f32 && cic == 2 && nout == 16) return launch_col_t<2, 16, false>(a, sms, st);
    if (out_f32 && cic == 4 && nout == 16) return launch_col_t<4, 16, true>(a, sms, st);
    if (out_f32 && cic == 2 && nout == 16) return launch_col_t<2, 16, true>(a, sms, st);
    return cudaErrorInvalidValue;
  }
  if (!out_f32 && cic == 2 && nout == 32) return launch_conv_t<2, 32, false>(a, sms, st);
  if (!out_f32 && cic == 4 && nout == 32) return launch_conv_t<4, 32, false>(a, sms, st);
  if (!out_f32 && cic == 2 && nout == 16) return launch_conv_t<2, 16, false>(a, sms, st);
  if (out_f32 && cic == 4 && nout == 16) return launch_conv_t<4, 16, true>(a, sms, st);
  if (out_f32 && cic == 2 && nout == 16) return launch_conv_t<2, 16, true>(a, sms, st);
  return cudaErrorInvalidValue;
}

}  // namespace kp
