// kp_cnn.cu -- the learned initial guess: a small 3x3 convolutional network
// trained on the GPU by this library's own forward and backward kernels.
//
// Every convolution is an implicit GEMM on the tcgen05 tensor cores (the
// projection GEMM of kp_proj_tc.cu, BF16 operands, FP32 accumulation):
//   forward      Z[p][co]   = sum_k Xcol[p][k]  W[co][k]        k = c*9 + tap
//   input grad   dX[p][c]   = sum_k dZcol[p][k] W2[c][k]        k = co*9 + tap
//   weight grad  dW[co][k]  = sum_p dZt[co][p]  XcolT[k][p]     (split over p)
// with im2col gathers (zero padding at the grid border) writing the BF16
// operands.  Biases, ReLU, the MSE loss and Adam (FP32 master weights, BF16
// copies for the tensor cores) are elementwise kernels.  Activations are FP32
// planes [B][C][H*W] in the solver's y-fastest order.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "kp.h"
#include "kp_ctx.h"
#include "kp_dd.cuh"
#include "kp_internal.cuh"

namespace {

using kp::dd;
using kp::dd_add;
using kp::dd_add_f;
using kp::dd_from_double;
using kp::dd_mul;
using kp::dd_sub;
using kp::dd_to_double;
using kp::f32_nearest;

constexpr int kMaxLayers = 8;

__device__ __forceinline__ int tap_offset(int tap, int H) {   // (di, dj) in {-1,0,1}^2
  const int di = tap / 3 - 1, dj = tap % 3 - 1;
  return di * H + dj;
}

__device__ __forceinline__ bool tap_inside(int pp, int tap, int H, int W, int sign) {
  const int i = pp / H, j = pp - i * H;
  const int di = sign * (tap / 3 - 1), dj = sign * (tap % 3 - 1);
  return (unsigned)(i + di) < (unsigned)W && (unsigned)(j + dj) < (unsigned)H;
}

// Xcol[b*P + p][c*9 + tap] = X[b][c][p + sign*off(tap)] (0 outside the grid)
__global__ void im2col_kernel(const float* X, __nv_bfloat16* Xcol, int ld, int C, int H, int W, int sign) {
  const int P = H * W;
  const size_t row = blockIdx.x;                 // b*P + p
  const int b = (int)(row / P), p = (int)(row - (size_t)b * P);
  for (int k = threadIdx.x; k < ld; k += blockDim.x) {
    float v = 0.f;
    if (k < 9 * C) {
      const int c = k / 9, tap = k - c * 9;
      if (tap_inside(p, tap, H, W, sign)) v = X[((size_t)b * C + c) * P + p + sign * tap_offset(tap, H)];
    }
    Xcol[row * ld + k] = __float2bfloat16_rn(v);
  }
}

// XcolT[c*9 + tap][b*P + p] = X[b][c][p + off(tap)]
__global__ void im2colT_kernel(const float* X, __nv_bfloat16* XcolT, size_t ld, int C, int H, int W, int B) {
  const int P = H * W;
  const int k = blockIdx.y;                      // c*9 + tap
  const int c = k / 9, tap = k - c * 9;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < (size_t)B * P;
       q += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(q / P), p = (int)(q - (size_t)b * P);
    float v = 0.f;
    if (tap_inside(p, tap, H, W, 1)) v = X[((size_t)b * C + c) * P + p + tap_offset(tap, H)];
    XcolT[(size_t)k * ld + q] = __float2bfloat16_rn(v);
  }
}

// dZt[co][b*P + p] = dZ[b][co][p]
__global__ void planes_to_rows_kernel(const float* dZ, __nv_bfloat16* dZt, size_t ld, int C, int P, int B) {
  const int co = blockIdx.y;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < (size_t)B * P;
       q += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(q / P), p = (int)(q - (size_t)b * P);
    dZt[(size_t)co * ld + q] = __float2bfloat16_rn(dZ[((size_t)b * C + co) * P + p]);
  }
}

// Y[b][co][p] = act(Cm[b*P + p][co] + bias[co])
__global__ void fwd_epilogue_kernel(const float* Cm, int ldc, const float* bias, float* Y, int Cout, int P,
                                    int B, int relu) {
  const size_t n = (size_t)B * Cout * P;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(q % P);
    const size_t bc = q / P;
    const int co = (int)(bc % Cout), b = (int)(bc / Cout);
    float v = Cm[((size_t)b * P + p) * ldc + co] + bias[co];
    Y[q] = relu ? fmaxf(v, 0.f) : v;
  }
}

// dZprev[b][c][p] = (Yprev > 0) * Cm[b*P + p][c]  (input gradient through ReLU)
__global__ void dgrad_epilogue_kernel(const float* Cm, int ldc, const float* Yprev, float* dZprev, int Cin,
                                      int P, int B) {
  const size_t n = (size_t)B * Cin * P;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    const int p = (int)(q % P);
    const size_t bc = q / P;
    const int c = (int)(bc % Cin), b = (int)(bc / Cin);
    dZprev[q] = Yprev[q] > 0.f ? Cm[((size_t)b * P + p) * ldc + c] : 0.f;
  }
}

// MSE loss over B*P values and its gradient 2 (y - t) / (B P)
__global__ void mse_kernel(const float* y, const float* t, float* dz, size_t n, double* loss) {
  __shared__ double red[256];
  double s = 0.0;
  const float sc = 2.f / (float)n;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    const float d = y[q] - t[q];
    dz[q] = sc * d;
    s += (double)d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] / (double)n);
}

// db[co] += sum over b, p of dZ[b][co][p]
__global__ void bias_grad_kernel(const float* dZ, float* db, int Cout, int P, int B) {
  __shared__ float red[256];
  const int co = blockIdx.y;
  float s = 0.f;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < (size_t)B * P;
       q += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(q / P), p = (int)(q - (size_t)b * P);
    s += dZ[((size_t)b * Cout + co) * P + p];
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(db + co, red[0]);
}

// Adam on the FP32 master parameters (Kingma & Ba 2015)
__global__ void adam_kernel(float* w, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const float gq = g[q];
    const float mq = b1 * m[q] + (1.f - b1) * gq;
    const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
    m[q] = mq;
    v[q] = vq;
    w[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
  }
}

// BF16 tensor-core copies of layer weights: Wb[co][k] (k = c*9+tap) and the
// transposed W2b[c][k'] (k' = co*9+tap) used by the input gradient
__global__ void weights_bf16_kernel(const float* Wl, __nv_bfloat16* Wb, int ldw, __nv_bfloat16* W2b, int ldw2,
                                    int Cin, int Cout) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < Cout * Cin * 9; q += gridDim.x * blockDim.x) {
    const int co = q / (Cin * 9), k = q - co * Cin * 9;
    const int c = k / 9, tap = k - c * 9;
    const __nv_bfloat16 v = __float2bfloat16_rn(Wl[q]);
    Wb[(size_t)co * ldw + k] = v;
    W2b[(size_t)c * ldw2 + co * 9 + tap] = v;
  }
}

size_t up8(size_t x) { return (x + 7) / 8 * 8; }

// A field as two BF16 operands: hi = bf16(f), lo = bf16(256 (f - hi)) of its
// FP32 value f.  One BF16 plane holds 8 significant bits; the step's change the
// network predicts is a difference of neighbours a few hundred times smaller
// than m, so the first layer gets both planes (about 16 bits) and recombines
// them in its FP32 sums.  f - hi is exact in FP32 (both are multiples of f's
// ulp and |f - hi| is at most half a BF16 ulp of f), so the split costs FP32
// arithmetic only; from the FP64 field it differs from splitting m itself only
// where 256 (f - hi) is a BF16 rounding tie (one lo ulp, 2^-17 of m).
__device__ __forceinline__ void split_hi_lo(float f, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(f);
  lo = __float2bfloat16_rn((f - __bfloat162float(hi)) * 256.f);
}

// The residual the step leaves at the image, r = m/dt - A(m~ = m) m at point
// p (Sec. 2.3, f = 0, zero outside the grid).  With A m = (1/dt + 4c) m_p +
// sum over the four neighbours of (-c -+ e (m_+ - m_-)) m_nbr, the 1/dt terms
// cancel exactly and the rest collects into
//   r = c (m_E + m_W + m_N + m_S - 4 m_p) + e ((m_E - m_W)^2 + (m_N - m_S)^2),
// c = g2/(2h^2) = g2 H^2 / 2, e = g2 H^2 / 8 -- no division, and none of the
// cancellation of the two large 1/dt terms.  Evaluated in double-float on the
// FP32 pipe (kp_dd.cuh; about 2^-44 of c |m| absolute), the FP64 field split
// without FP64 instructions.
__device__ __forceinline__ dd step_residual_at(const double* m, int p, int H, int W, dd c, dd e) {
  const int i = p / H, j = p - i * H;
  const dd z = {0.f, 0.f};
  const dd mC = dd_from_double(m[p]);
  const dd mE = i + 1 < W ? dd_from_double(m[p + H]) : z, mW = i > 0 ? dd_from_double(m[p - H]) : z;
  const dd mN = j + 1 < H ? dd_from_double(m[p + 1]) : z, mS = j > 0 ? dd_from_double(m[p - 1]) : z;
  const dd lap = dd_sub(dd_add(dd_add(mE, mW), dd_add(mN, mS)), dd{4.f * mC.hi, 4.f * mC.lo});
  const dd dx = dd_sub(mE, mW), dy = dd_sub(mN, mS);
  return dd_add(dd_mul(c, lap), dd_mul(e, dd_add(dd_mul(dx, dx), dd_mul(dy, dy))));
}

// rho_b = ||r_b|| / sqrt(P), one block per sample; g2 = g2v, or g2s[*step +
// step_offset] when g2s is given (the march's schedule and counter).  The FP32
// value of r goes to rout[b * rld + p] for the packing kernels.  The squares
// are summed in double-float per thread; no FP64 instruction runs per point
// (the FP64 pipe, not HBM, bounds this part on GB300).  Blocks of 1024
// threads: with one block per plane, fewer and larger blocks keep the last
// wave short (1536 planes are 5 waves of 2 blocks per SM, not 1.3 waves of 8).
constexpr int kRmsThreads = 1024;

__global__ void step_residual_rms_kernel(const double* const* m, int H, int W, double dt, double g2v,
                                         const double* g2s, const int* step, int step_offset, double* rho,
                                         float* rout, size_t rld) {
  __shared__ double red[32];
  const int b = blockIdx.x, P = H * W;
  const double g2 = g2s ? g2s[*step + step_offset] : g2v;
  const double hh = (double)H * (double)H;
  const dd c = dd_from_double(0.5 * g2 * hh), e = dd_from_double(0.125 * g2 * hh);
  float* ro = rout + (size_t)b * rld;
  dd acc = {0.f, 0.f};
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    const dd r = step_residual_at(m[b], p, H, W, c, e);
    acc = dd_add(acc, dd_mul(r, r));
    ro[p] = r.hi;
  }
  double s = dd_to_double(acc);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    rho[b] = sqrt(t / P);
  }
}

// Network input planes of sample b: the target's plane (its lagged field
// m_i^{n-1} for the learned guess) and the seed state, each as its hi and lo
// planes, the time embedding tau, 1 - tau, sin(pi tau), cos(pi tau), and the
// step's residual at the target's plane scaled to unit rms (hi, lo).  Plane 8
// holds the FP32 residual on entry (step_residual_rms_kernel) and is
// overwritten by the same thread.
__global__ void pack_inputs_kernel(const double* const* img, const double* const* seed, float tau,
                                   const double* rho, int P, float* in) {
  const int b = blockIdx.y;
  const float e[4] = {tau, 1.f - tau, sinpif(tau), cospif(tau)};
  const float ir = rho[b] > 0.0 ? 1.f / f32_nearest(rho[b]) : 0.f;
  float* o = in + (size_t)b * 10 * P;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    __nv_bfloat16 h0, l0, h1, l1, h2, l2;
    split_hi_lo(f32_nearest(img[b][p]), h0, l0);
    split_hi_lo(f32_nearest(seed[b][p]), h1, l1);
    split_hi_lo(o[8 * P + p] * ir, h2, l2);
    o[p] = __bfloat162float(h0);
    o[P + p] = __bfloat162float(l0);
    o[2 * P + p] = __bfloat162float(h1);
    o[3 * P + p] = __bfloat162float(l1);
#pragma unroll
    for (int k = 0; k < 4; ++k) o[(4 + k) * P + p] = e[k];
    o[8 * P + p] = __bfloat162float(h2);
    o[9 * P + p] = __bfloat162float(l2);
  }
}

// out_b = (a_b - b_b) * scale / rho_b in FP32 (training targets
// (m_i^n - m_i^{n-1}) / (dt rho_b); rho NULL = 1)
__global__ void diff_kernel(const double* const* a, const double* const* bb, const double* rho, double scale,
                            float* out, int P) {
  const int b = blockIdx.y;
  const double s = rho ? (rho[b] > 0.0 ? scale / rho[b] : 0.0) : scale;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x)
    out[(size_t)b * P + p] = (float)((a[b][p] - bb[b][p]) * s);
}

// x_b = base_b + scale * rho_b * delta_b (FP64 initial guess from the
// network's output; rho NULL = 1)
__global__ void add_guess_kernel(const float* delta, const double* const* base, const double* rho, double scale,
                                 double* const* x, int P) {
  const int b = blockIdx.y;
  const double s = rho ? scale * rho[b] : scale;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x)
    x[b][p] = base[b][p] + s * (double)delta[(size_t)b * P + p];
}

// The learned guess inside the time march, for the target timestep n = *step
// + step_offset + 1 (1-based), tau = n / T: the ten input planes of sample b
// -- m_i^{n-1} (hi, lo), m_seed^n (hi, lo), tau, 1 - tau, sin pi tau,
// cos pi tau, the step's residual (FP32 in r, step_residual_rms_kernel)
// scaled by 1 / rho_b (hi, lo) -- straight into the padded BF16 rows of the
// first convolution (chunk 0: channels 0..7; chunk 1: 8, 9 and zeros)
__global__ void march_pack_kernel(const double* const* mprev, const double* const* mseed, const float* r,
                                  const int* step, int step_offset, const double* rho, int T, int H, int W,
                                  int halo, int Rp, __nv_bfloat16* out) {
  const int b = blockIdx.y;
  const int P = H * W;
  const int t = *step + step_offset;
  const float tau = (float)(t + 1) / (float)T;
  const float e[4] = {tau, 1.f - tau, sinpif(tau), cospif(tau)};
  const float ir = rho[b] > 0.0 ? 1.f / f32_nearest(rho[b]) : 0.f;
  const double* mp = mprev[b];
  const double* ms = mseed[b];
  const float* rb = r + (size_t)b * P;
  __nv_bfloat162 h1 = __floats2bfloat162_rn(e[0], e[1]);
  __nv_bfloat162 h2 = __floats2bfloat162_rn(e[2], e[3]);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    const int i = p / H, j = p - i * H;
    const size_t row = (size_t)halo + (size_t)i * (H + 2) + 1 + j;
    __nv_bfloat162 f0, f1, f2;
    split_hi_lo(f32_nearest(mp[p]), f0.x, f0.y);
    split_hi_lo(f32_nearest(ms[p]), f1.x, f1.y);
    split_hi_lo(rb[p] * ir, f2.x, f2.y);
    const uint4 c0 = make_uint4(*reinterpret_cast<uint32_t*>(&f0), *reinterpret_cast<uint32_t*>(&f1),
                                *reinterpret_cast<uint32_t*>(&h1), *reinterpret_cast<uint32_t*>(&h2));
    *reinterpret_cast<uint4*>(out + (((size_t)b * 2 + 0) * Rp + row) * 8) = c0;
    *reinterpret_cast<uint4*>(out + (((size_t)b * 2 + 1) * Rp + row) * 8) =
        make_uint4(*reinterpret_cast<uint32_t*>(&f2), 0u, 0u, 0u);
  }
}


}  // namespace

struct kp_cnn {
  kp_ctx* ctx = nullptr;
  int H = 0, W = 0, P = 0, maxB = 0, L = 0;
  int ch[kMaxLayers + 1] = {0};
  std::vector<size_t> woff, boff;      // offsets of W[l] and b[l] in the flat parameter array
  int nparams = 0;
  float* params = nullptr;             // FP32 master [nparams]
  float* grads = nullptr;
  float* adam_m = nullptr;
  float* adam_v = nullptr;
  __nv_bfloat16* wb = nullptr;         // per layer Wb then W2b, packed
  std::vector<size_t> wb_off, w2b_off;
  float* act = nullptr;                // Y[l] for l = 1..L, packed
  std::vector<size_t> act_off;
  float* dz = nullptr;                 // [maxB][Cmax][P]
  float* dz2 = nullptr;
  __nv_bfloat16* col = nullptr;        // im2col rows [maxB*P][ldmax]
  __nv_bfloat16* colT = nullptr;       // [9*Cmax][maxB*P]
  __nv_bfloat16* rows = nullptr;       // [Cmax][maxB*P]
  float* cm = nullptr;                 // GEMM output [maxB*P][48]
  kp::ProjTile* tiles = nullptr;
  size_t tiles_cap = 0;
  double* d_loss = nullptr;
  int* d_err = nullptr;
  int Cmax = 0;
  // inference on the implicit-GEMM convolutions of kp_conv_tc.cu (no im2col
  // in memory): input <= 16 channels (2 chunks of 8), hidden layers <= 32
  // (4 chunks), output <= 16 (MMA N = 16)
  bool fused = false;
  kp::ConvGeom geo{};
  __nv_bfloat16* pin = nullptr;                 // [maxB][2][Rp][8]
  __nv_bfloat16* px[2] = {nullptr, nullptr};    // [maxB][4][Rp][8], alternating layers
  __nv_bfloat16* wf = nullptr;                  // per layer [9][cic][nout][8]
  std::vector<size_t> wf_off;
  std::vector<int> cic, nout;
  int infB = 0;                                 // images the inference buffers hold
  float* dout = nullptr;                        // [infB][P] network output (march guesses)
  double* rho = nullptr;                        // [max(infB, maxB)] rms of each sample's step residual
};

namespace {

kp_status gemm(kp_cnn* n, const __nv_bfloat16* Bop, int brows, int K, size_t ldb,
               const __nv_bfloat16* Vop, int vrows, size_t ldv, float* C, int ldc,
               const std::vector<kp::ProjTile>& tiles) {
  kp_ctx* c = n->ctx;
  alignas(64) CUtensorMap mb, mv;
  cudaError_t e = kp::make_bf16_map(&mb, Bop, brows, K, (int)ldb, 128);
  if (e == cudaSuccess) e = kp::make_bf16_map(&mv, Vop, vrows, K, (int)ldv, 48);
  if (e == cudaSuccess && tiles.size() > n->tiles_cap) {
    cudaFree(n->tiles);
    n->tiles = nullptr;
    e = cudaMalloc((void**)&n->tiles, tiles.size() * sizeof(kp::ProjTile));
    n->tiles_cap = e == cudaSuccess ? tiles.size() : 0;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(n->tiles, tiles.data(), tiles.size() * sizeof(kp::ProjTile), cudaMemcpyHostToDevice,
                        c->stream);
  if (e == cudaSuccess)
    e = kp::launch_proj_gemm_bf16(mb, mv, n->tiles, (int)tiles.size(), K, C, ldc, n->d_err,
                                  std::min((int)tiles.size(), c->sms), c->stream);
  return e == cudaSuccess ? KP_OK : kp::cuda_error(c, e, "CNN GEMM");
}

// Tiles of 128 rows of the B operand against one 48-row tile of V.
std::vector<kp::ProjTile> row_tiles(int rows, int nv) {
  std::vector<kp::ProjTile> t;
  for (int r = 0; r < rows; r += 128) {
    kp::ProjTile x{};
    x.row0 = r; x.vrow0 = 0; x.crow0 = r; x.count = std::min(128, rows - r); x.nv = nv;
    t.push_back(x);
  }
  return t;
}

int grid_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 4096); }

kp_status forward_impl(kp_cnn* n, int B, const float* in) {
  cudaStream_t st = n->ctx->stream;
  const int P = n->P;
  const float* X = in;
  for (int l = 0; l < n->L; ++l) {
    const int cin = n->ch[l], cout = n->ch[l + 1];
    const size_t ld = up8(9 * cin);
    im2col_kernel<<<B * P, 64, 0, st>>>(X, n->col, (int)ld, cin, n->H, n->W, 1);
    kp_status s = gemm(n, n->col, B * P, 9 * cin, ld, n->wb + n->wb_off[l], cout, ld, n->cm, 48,
                       row_tiles(B * P, cout));
    if (s != KP_OK) return s;
    float* Y = n->act + n->act_off[l];
    fwd_epilogue_kernel<<<grid_for((size_t)B * cout * P), 256, 0, st>>>(
        n->cm, 48, n->params + n->boff[l], Y, cout, P, B, l + 1 < n->L);
    X = Y;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KP_OK : kp::cuda_error(n->ctx, e, "CNN forward");
}

kp_status refresh_bf16(kp_cnn* n) {
  cudaStream_t st = n->ctx->stream;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l < n->L; ++l) {
    const int cin = n->ch[l], cout = n->ch[l + 1];
    weights_bf16_kernel<<<grid_for((size_t)cout * cin * 9), 256, 0, st>>>(
        n->params + n->woff[l], n->wb + n->wb_off[l], (int)up8(9 * cin), n->wb + n->w2b_off[l],
        (int)up8(9 * cout), cin, cout);
    if (n->fused && e == cudaSuccess)
      e = kp::launch_conv_weights(n->params + n->woff[l], cin, cout, n->cic[l], n->nout[l], n->wf + n->wf_off[l], st);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  return e == cudaSuccess ? KP_OK : kp::cuda_error(n->ctx, e, "CNN weights");
}

// The layers of the implicit-GEMM inference from the packed input rows in
// n->pin: one convolution launch per layer, the last writing FP32 planes.
cudaError_t conv_layers(kp_cnn* n, int B, float* out, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  const __nv_bfloat16* X = n->pin;
  for (int l = 0; l < n->L && e == cudaSuccess; ++l) {
    const bool last = l + 1 == n->L;
    __nv_bfloat16* Y = last ? nullptr : n->px[l & 1];
    e = kp::launch_conv3x3(X, B, n->cic[l], n->wf + n->wf_off[l], n->params + n->boff[l], n->ch[l + 1],
                           n->nout[l], n->geo, Y, last ? out : nullptr, n->d_err, n->ctx->sms, st);
    X = Y;
  }
  return e;
}

// Inference: input planes -> padded BF16 rows, then the layers.
kp_status forward_fused(kp_cnn* n, int B, const float* in, float* out) {
  cudaStream_t st = n->ctx->stream;
  cudaError_t e = kp::launch_planes_to_padded(in, B, n->ch[0], 2, n->geo, n->pin, st);
  if (e == cudaSuccess) e = conv_layers(n, B, out, st);
  return e == cudaSuccess ? KP_OK : kp::cuda_error(n->ctx, e, "CNN forward (implicit GEMM)");
}

// (Re)allocate the implicit-GEMM inference buffers for B images, zeroed (the
// padding rows are never written afterwards).
cudaError_t alloc_inference(kp_cnn* n, int B) {
  cudaFree(n->pin); cudaFree(n->px[0]); cudaFree(n->px[1]); cudaFree(n->dout); cudaFree(n->rho);
  n->pin = n->px[0] = n->px[1] = nullptr;
  n->dout = nullptr;
  n->rho = nullptr;
  n->infB = 0;
  const size_t rows = (size_t)B * n->geo.Rp * 8;
  cudaError_t e = cudaMalloc((void**)&n->pin, 2 * rows * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMemset(n->pin, 0, 2 * rows * sizeof(__nv_bfloat16));
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaMalloc((void**)&n->px[k], 4 * rows * sizeof(__nv_bfloat16));
    if (e == cudaSuccess) e = cudaMemset(n->px[k], 0, 4 * rows * sizeof(__nv_bfloat16));
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->dout, (size_t)B * n->P * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->rho, (size_t)std::max(B, n->maxB) * sizeof(double));
  if (e == cudaSuccess) n->infB = B;
  return e;
}

// forward + MSE + backward into n->grads; loss on the host if wanted
kp_status backward_impl(kp_cnn* n, int B, const float* in, const float* target, double* loss) {
  cudaStream_t st = n->ctx->stream;
  const int P = n->P;
  kp_status s = forward_impl(n, B, in);
  if (s != KP_OK) return s;
  cudaError_t e = cudaMemsetAsync(n->grads, 0, (size_t)n->nparams * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->d_loss, 0, sizeof(double), st);
  if (e != cudaSuccess) return kp::cuda_error(n->ctx, e, "CNN backward");
  const size_t nout = (size_t)B * P;
  mse_kernel<<<grid_for(nout), 256, 0, st>>>(n->act + n->act_off[n->L - 1], target, n->dz, nout, n->d_loss);
  float* dZ = n->dz;
  float* dZo = n->dz2;
  const size_t ldp = up8((size_t)B * P);
  for (int l = n->L - 1; l >= 0; --l) {
    const int cin = n->ch[l], cout = n->ch[l + 1];
    const float* X = l == 0 ? in : n->act + n->act_off[l - 1];
    // bias gradient
    bias_grad_kernel<<<dim3(64, cout), 256, 0, st>>>(dZ, n->grads + n->boff[l], cout, P, B);
    // weight gradient: dW[co][k] = sum_p dZt[co][p] XcolT[k][p], split over p
    im2colT_kernel<<<dim3(grid_for((size_t)B * P), 9 * cin), 256, 0, st>>>(X, n->colT, ldp, cin, n->H, n->W, B);
    planes_to_rows_kernel<<<dim3(grid_for((size_t)B * P), cout), 256, 0, st>>>(dZ, n->rows, ldp, cout, P, B);
    {
      std::vector<kp::ProjTile> tl;
      const int nk = (int)((B * (size_t)P + 63) / 64);
      const int ntn = (9 * cin + 47) / 48;
      const int splits = std::max(1, std::min(nk, (2 * n->ctx->sms) / std::max(ntn, 1)));
      for (int tn = 0; tn < ntn; ++tn)
        for (int sp = 0; sp < splits; ++sp) {
          kp::ProjTile t{};
          t.row0 = 0; t.vrow0 = 48 * tn; t.crow0 = 0; t.count = cout;
          t.nv = std::min(48, 9 * cin - 48 * tn); t.ccol0 = 48 * tn;
          t.kc0 = (int)((long long)nk * sp / splits); t.kc1 = (int)((long long)nk * (sp + 1) / splits);
          t.atomic = 1;
          if (t.kc1 > t.kc0) tl.push_back(t);
        }
      s = gemm(n, n->rows, cout, B * P, ldp, n->colT, 9 * cin, ldp, n->grads + n->woff[l], 9 * cin, tl);
      if (s != KP_OK) return s;
    }
    if (l == 0) break;
    // input gradient through the previous layer's ReLU
    const size_t ld2 = up8(9 * cout);
    im2col_kernel<<<B * P, 64, 0, st>>>(dZ, n->col, (int)ld2, cout, n->H, n->W, -1);
    s = gemm(n, n->col, B * P, 9 * cout, ld2, n->wb + n->w2b_off[l], cin, ld2, n->cm, 48, row_tiles(B * P, cin));
    if (s != KP_OK) return s;
    dgrad_epilogue_kernel<<<grid_for((size_t)B * cin * P), 256, 0, st>>>(n->cm, 48, n->act + n->act_off[l - 1],
                                                                          dZo, cin, P, B);
    std::swap(dZ, dZo);
  }
  e = cudaGetLastError();
  if (e == cudaSuccess && loss) {
    e = cudaMemcpyAsync(loss, n->d_loss, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  return e == cudaSuccess ? KP_OK : kp::cuda_error(n->ctx, e, "CNN backward");
}

}  // namespace

extern "C" {

kp_status kp_cnn_destroy(kp_cnn* n) {
  if (!n) return KP_OK;
  if (n->ctx) cudaStreamSynchronize(n->ctx->stream);
  cudaFree(n->params); cudaFree(n->grads); cudaFree(n->adam_m); cudaFree(n->adam_v); cudaFree(n->wb);
  cudaFree(n->act); cudaFree(n->dz); cudaFree(n->dz2); cudaFree(n->col); cudaFree(n->colT); cudaFree(n->rows);
  cudaFree(n->cm); cudaFree(n->tiles); cudaFree(n->d_loss); cudaFree(n->d_err);
  cudaFree(n->pin); cudaFree(n->px[0]); cudaFree(n->px[1]); cudaFree(n->wf); cudaFree(n->dout);
  cudaFree(n->rho);
  delete n;
  return KP_OK;
}

kp_status kp_cnn_create(kp_ctx* c, int H, int W, int max_batch, int nlayers, const int* channels,
                        kp_cnn** out) {
  if (!c) return KP_ERR_ARG;
  if (!out || H < 1 || W < 1 || max_batch < 1 || nlayers < 1 || nlayers > kMaxLayers || !channels)
    return kp::set_error(c, KP_ERR_ARG, "CNN: bad sizes");
  for (int l = 0; l <= nlayers; ++l)
    if (channels[l] < 1 || channels[l] > 32) return kp::set_error(c, KP_ERR_ARG, "CNN: 1..32 channels per layer");
  if ((size_t)max_batch * H * W > (1u << 30)) return kp::set_error(c, KP_ERR_ARG, "CNN: batch too large");
  kp_cnn* n = new kp_cnn();
  n->ctx = c; n->H = H; n->W = W; n->P = H * W; n->maxB = max_batch; n->L = nlayers;
  for (int l = 0; l <= nlayers; ++l) { n->ch[l] = channels[l]; n->Cmax = std::max(n->Cmax, channels[l]); }
  size_t np = 0, nwb = 0, nact = 0;
  for (int l = 0; l < nlayers; ++l) {
    const int cin = n->ch[l], cout = n->ch[l + 1];
    n->woff.push_back(np); np += (size_t)cout * cin * 9;
    n->boff.push_back(np); np += cout;
    n->wb_off.push_back(nwb); nwb += (size_t)cout * up8(9 * cin);
    nwb = up8(nwb);
    n->w2b_off.push_back(nwb); nwb += (size_t)cin * up8(9 * cout);
    nwb = up8(nwb);
    n->act_off.push_back(nact); nact += (size_t)max_batch * cout * n->P;
  }
  n->nparams = (int)np;
  const size_t BP = (size_t)max_batch * n->P;
  const size_t ldmax = up8(9 * n->Cmax);
  cudaError_t e = cudaMalloc((void**)&n->params, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->grads, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->adam_m, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->adam_v, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->wb, nwb * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMemset(n->wb, 0, nwb * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->act, nact * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->dz, BP * n->Cmax * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->dz2, BP * n->Cmax * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->col, BP * ldmax * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->colT, 9 * (size_t)n->Cmax * up8(BP) * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->rows, (size_t)n->Cmax * up8(BP) * sizeof(__nv_bfloat16));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->cm, BP * 48 * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->d_loss, sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&n->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(n->d_err, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(n->params, 0, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->adam_m, 0, np * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(n->adam_v, 0, np * sizeof(float));
  // implicit-GEMM inference buffers (zero rows stay zero: never written)
  n->fused = nlayers >= 2 && n->ch[0] <= 16 && n->ch[nlayers] <= 16;
  n->geo = kp::conv_geom(H, W);
  size_t nwf = 0;
  for (int l = 0; l < nlayers; ++l) {
    // input chunk planes (8 channels each, K = 16 per MMA) and output width
    n->cic.push_back(l == 0 || n->ch[l] <= 16 ? 2 : 4);
    n->nout.push_back(l + 1 == nlayers || n->ch[l + 1] <= 16 ? 16 : 32);
    n->wf_off.push_back(nwf);
    nwf += (size_t)9 * n->cic[l] * n->nout[l] * 8;
    if (kp::conv_smem_bytes(n->geo, n->cic[l], n->nout[l]) > c->smem_optin) n->fused = false;
  }
  if (n->fused && e == cudaSuccess) {
    e = alloc_inference(n, max_batch);
    if (e == cudaSuccess) e = cudaMalloc((void**)&n->wf, nwf * sizeof(__nv_bfloat16));
  }
  if (e != cudaSuccess) {
    kp_status r = kp::cuda_error(c, e, "CNN allocation");
    kp_cnn_destroy(n);
    return r;
  }
  *out = n;
  return KP_OK;
}

int kp_cnn_num_params(const kp_cnn* n) { return n ? n->nparams : 0; }

kp_status kp_cnn_set_params(kp_cnn* n, const float* host) {
  if (!n || !host) return KP_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(n->params, host, (size_t)n->nparams * sizeof(float), cudaMemcpyHostToDevice,
                                  n->ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->adam_m, 0, (size_t)n->nparams * sizeof(float), n->ctx->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(n->adam_v, 0, (size_t)n->nparams * sizeof(float), n->ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->ctx->stream);
  if (e != cudaSuccess) return kp::cuda_error(n->ctx, e, "CNN parameters");
  return refresh_bf16(n);
}

kp_status kp_cnn_get_params(kp_cnn* n, float* host) {
  if (!n || !host) return KP_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(host, n->params, (size_t)n->nparams * sizeof(float), cudaMemcpyDeviceToHost,
                                  n->ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(n->ctx->stream);
  return e == cudaSuccess ? KP_OK : kp::cuda_error(n->ctx, e, "CNN parameters");
}

kp_status kp_cnn_set_inference_batch(kp_cnn* n, int B) {
  if (!n) return KP_ERR_ARG;
  if (B < 1 || (size_t)B * n->P > (1u << 30)) return kp::set_error(n->ctx, KP_ERR_ARG, "CNN: bad inference batch");
  if (!n->fused) return kp::set_error(n->ctx, KP_ERR_UNSUPPORTED, "CNN: no implicit-GEMM inference for this shape");
  cudaError_t e = cudaStreamSynchronize(n->ctx->stream);   // no launch still reads the old buffers
  if (e == cudaSuccess) e = alloc_inference(n, B);
  return e == cudaSuccess ? KP_OK : kp::cuda_error(n->ctx, e, "CNN inference buffers");
}

kp_status kp_cnn_forward(kp_cnn* n, int B, const float* in, float* out) {
  if (!n || B < 1 || !in || !out) return n ? kp::set_error(n->ctx, KP_ERR_ARG, "CNN forward: bad batch") : KP_ERR_ARG;
  if (n->fused) {
    if (B > n->infB) return kp::set_error(n->ctx, KP_ERR_ARG, "CNN forward: batch above the inference batch %d", n->infB);
    return forward_fused(n, B, in, out);
  }
  if (B > n->maxB) return kp::set_error(n->ctx, KP_ERR_ARG, "CNN forward: bad batch");
  kp_status s = forward_impl(n, B, in);
  if (s != KP_OK) return s;
  cudaError_t e = cudaMemcpyAsync(out, n->act + n->act_off[n->L - 1], (size_t)B * n->P * n->ch[n->L] * sizeof(float),
                                  cudaMemcpyDeviceToDevice, n->ctx->stream);
  return e == cudaSuccess ? KP_OK : kp::cuda_error(n->ctx, e, "CNN forward");
}

kp_status kp_cnn_gradients(kp_cnn* n, int B, const float* in, const float* target, float* grads, double* loss) {
  if (!n || B < 1 || B > n->maxB || !in || !target) return n ? kp::set_error(n->ctx, KP_ERR_ARG, "CNN: bad batch") : KP_ERR_ARG;
  if (n->ch[n->L] != 1) return kp::set_error(n->ctx, KP_ERR_UNSUPPORTED, "CNN: loss needs one output channel");
  kp_status s = backward_impl(n, B, in, target, loss);
  if (s != KP_OK || !grads) return s;
  cudaError_t e = cudaMemcpyAsync(grads, n->grads, (size_t)n->nparams * sizeof(float), cudaMemcpyDeviceToDevice,
                                  n->ctx->stream);
  return e == cudaSuccess ? KP_OK : kp::cuda_error(n->ctx, e, "CNN gradients");
}

kp_status kp_cnn_pack_inputs(kp_cnn* n, int B, const double* const* img, const double* const* seed, int step,
                             int T, double g2n, float* in, double* rho) {
  if (!n || B < 1 || !img || !seed || !in || !rho || T < 1 || step < 1 || step > T || !(g2n >= 0.0))
    return n ? kp::set_error(n->ctx, KP_ERR_ARG, "CNN pack: bad arguments") : KP_ERR_ARG;
  if (n->ch[0] != 10) return kp::set_error(n->ctx, KP_ERR_UNSUPPORTED, "CNN pack: the network needs 10 input planes");
  std::vector<const double*> h(2 * (size_t)B);
  for (int b = 0; b < B; ++b) { h[b] = img[b]; h[B + b] = seed[b]; }
  const double** d = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d, h.size() * sizeof(double*), n->ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double*), cudaMemcpyHostToDevice, n->ctx->stream);
  if (e == cudaSuccess) {
    const double dt = 1.0 / T;
    step_residual_rms_kernel<<<B, kRmsThreads, 0, n->ctx->stream>>>(d, n->H, n->W, dt, g2n, nullptr, nullptr, 0, rho,
                                                            in + 8 * (size_t)n->P, 10 * (size_t)n->P);
    pack_inputs_kernel<<<dim3(grid_for(n->P), B), 256, 0, n->ctx->stream>>>(d, d + B, (float)step / (float)T,
                                                                           rho, n->P, in);
    e = cudaGetLastError();
  }
  if (d) cudaFreeAsync(d, n->ctx->stream);
  return e == cudaSuccess ? KP_OK : kp::cuda_error(n->ctx, e, "CNN pack");
}

kp_status kp_cnn_add_guess(kp_cnn* n, int B, const float* delta, const double* const* base, const double* rho,
                           double scale, double* const* x) {
  if (!n || B < 1 || !delta || !base || !x) return n ? kp::set_error(n->ctx, KP_ERR_ARG, "CNN guess: bad arguments") : KP_ERR_ARG;
  std::vector<const double*> h(2 * (size_t)B);
  for (int b = 0; b < B; ++b) { h[b] = base[b]; h[B + b] = x[b]; }
  const double** d = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d, h.size() * sizeof(double*), n->ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double*), cudaMemcpyHostToDevice, n->ctx->stream);
  if (e == cudaSuccess) {
    add_guess_kernel<<<dim3(grid_for(n->P), B), 256, 0, n->ctx->stream>>>(delta, d, rho, scale,
                                                                         const_cast<double* const*>(d + B), n->P);
    e = cudaGetLastError();
  }
  if (d) cudaFreeAsync(d, n->ctx->stream);
  return e == cudaSuccess ? KP_OK : kp::cuda_error(n->ctx, e, "CNN guess");
}

kp_status kp_cnn_pack_target(kp_cnn* n, int B, const double* const* a, const double* const* b, const double* rho,
                             double scale, float* out) {
  if (!n || B < 1 || !a || !b || !out) return n ? kp::set_error(n->ctx, KP_ERR_ARG, "CNN target: bad arguments") : KP_ERR_ARG;
  std::vector<const double*> h(2 * (size_t)B);
  for (int k = 0; k < B; ++k) { h[k] = a[k]; h[B + k] = b[k]; }
  const double** d = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&d, h.size() * sizeof(double*), n->ctx->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d, h.data(), h.size() * sizeof(double*), cudaMemcpyHostToDevice, n->ctx->stream);
  if (e == cudaSuccess) {
    diff_kernel<<<dim3(grid_for(n->P), B), 256, 0, n->ctx->stream>>>(d, d + B, rho, scale, out, n->P);
    e = cudaGetLastError();
  }
  if (d) cudaFreeAsync(d, n->ctx->stream);
  return e == cudaSuccess ? KP_OK : kp::cuda_error(n->ctx, e, "CNN target");
}

kp_status kp_cnn_train_step(kp_cnn* n, int B, const float* in, const float* target, float lr, float beta1,
                            float beta2, float eps, int t, double* loss) {
  if (!n || t < 1) return n ? kp::set_error(n->ctx, KP_ERR_ARG, "CNN: Adam step t >= 1") : KP_ERR_ARG;
  kp_status s = kp_cnn_gradients(n, B, in, target, nullptr, loss);
  if (s != KP_OK) return s;
  const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
  adam_kernel<<<grid_for(n->nparams), 256, 0, n->ctx->stream>>>(n->params, n->grads, n->adam_m, n->adam_v,
                                                                 n->nparams, lr, beta1, beta2, eps, c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return kp::cuda_error(n->ctx, e, "CNN Adam");
  return refresh_bf16(n);
}

}  // extern "C"

namespace kp {

bool cnn_march_ready(const kp_cnn* n, int H, int W) {
  return n && n->fused && n->H == H && n->W == W && n->ch[0] == 10 && n->ch[n->L] == 1 && n->infB > 0;
}

int cnn_inference_batch(const kp_cnn* n) { return n ? n->infB : 0; }

cudaError_t cnn_enqueue_guess(kp_cnn* n, int B, const double* const* mprev, const double* const* mseed,
                              float* delta, double* rho, const int* step, int step_offset, const double* g2,
                              int T, cudaStream_t st) {
  if (B < 1 || B > n->infB) return cudaErrorInvalidValue;
  const dim3 grid(std::min((n->P + 255) / 256, 1024), B);
  // the FP32 residual goes through the network's output buffer, which the
  // packing kernel has read before any layer runs
  step_residual_rms_kernel<<<B, kRmsThreads, 0, st>>>(mprev, n->H, n->W, 1.0 / T, 0.0, g2, step, step_offset, rho,
                                              n->dout, (size_t)n->P);
  march_pack_kernel<<<grid, 256, 0, st>>>(mprev, mseed, n->dout, step, step_offset, rho, T, n->H, n->W,
                                          n->geo.halo, n->geo.Rp, n->pin);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = conv_layers(n, B, delta, st);
  return e;
}

}  // namespace kp
