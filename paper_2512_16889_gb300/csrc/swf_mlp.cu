// Surrogate network for scans of the pair probability: a multilayer perceptron
//   (E, omega, lambda, p_x, p_y, s) -> 4 x [256, GELU] -> (mu, log sigma^2)
// trained on solver outputs.  BF16 operands on the tensor cores with FP32 accumulation
// (mma.sync m16n8k16), FP32 master weights, Adam, Gaussian negative log-likelihood
//   L = mean_b [ (y_b - mu_b)^2 exp(-l_b) + l_b ] / 2.
#include <cuda_bf16.h>

#include <cmath>
#include <map>
#include <cstring>
#include <string>
#include <vector>

#include "swf_internal.h"

namespace swf {
namespace mlp {

constexpr int NL = 5;                                // layers
constexpr int DIN[NL] = {6, 256, 256, 256, 256};
constexpr int DOUT[NL] = {256, 256, 256, 256, 2};

__host__ __device__ constexpr int n_params() {
  int n = 0;
  for (int l = 0; l < NL; ++l) n += DIN[l] * DOUT[l] + DOUT[l];
  return n;
}

// ---------------------------------------------------------------- BF16 GEMM (FP32 accumulate)
// C(m, n) = sum_k A(m, k) B(k, n); element (i, j) of a matrix X at X[i * sr + j * sc].
struct Mat {
  const __nv_bfloat16* p;
  long sr, sc;
};

enum Epi { EPI_FWD_HIDDEN = 0, EPI_FWD_OUT = 1, EPI_DX = 2, EPI_DW = 3 };

struct EpiArgs {
  int mode;
  const float* bias;          // FWD: [N]
  float* z;                   // FWD: pre-activation out [M][N]; DW: gradient out [M][N]
  __nv_bfloat16* act;         // FWD_HIDDEN: bf16 GELU(z) [M][N]; DX: bf16 dZ of the previous layer
  float* dz32;                // DX: fp32 dZ of the previous layer [M][N]
  const float* zprev;         // DX: pre-activation of the previous layer [M][N]
};

// The normal distribution function Phi(x) = (1 + erf(x / sqrt 2)) / 2 and the density phi(x),
// with erf from Abramowitz and Stegun's formula 7.1.26 (Hastings' rational approximation):
// erf(z) = 1 - (a1 t + a2 t^2 + a3 t^3 + a4 t^4 + a5 t^5) e^{-z^2}, t = 1/(1 + p z), z >= 0,
// |error| <= 1.5e-7.  One reciprocal, one exponential and five fused multiply-adds; the GELU
// values it gives are rounded to bfloat16 (8 significand bits) before use, far coarser than it.
__device__ __forceinline__ void normal_cdf_pdf(float x, float& cdf, float& pdf) {
  const float z = fabsf(x) * 0.70710678118654752f;
  const float t = __fdividef(1.0f, fmaf(0.3275911f, z, 1.0f));
  const float poly = t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f),
                                      -0.284496736f), 0.254829592f);
  const float e = __expf(-0.5f * x * x);  // e^{-z^2}
  const float tail = 0.5f * poly * e;     // (1 - erf(z)) / 2
  cdf = x >= 0.0f ? 1.0f - tail : tail;
  pdf = 0.39894228040143268f * e;
}
__device__ __forceinline__ float gelu(float x) {
  float c, d;
  normal_cdf_pdf(x, c, d);
  return x * c;
}
__device__ __forceinline__ float gelu_grad(float x) {
  float c, d;
  normal_cdf_pdf(x, c, d);
  return fmaf(x, d, c);
}

// The activation and its derivative elementwise (the network's own GELU, for checks).
__global__ void k_gelu_eval(const float* __restrict__ x, int n, float* __restrict__ g, float* __restrict__ dg) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    g[i] = gelu(x[i]);
    dg[i] = gelu_grad(x[i]);
  }
}

constexpr int TM = 64, TN = 64, TK = 16, SP = 24;  // tile, k step, padded smem row (bf16)

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) { return *reinterpret_cast<const uint32_t*>(p); }

__global__ void __launch_bounds__(128) k_gemm(Mat A, Mat B, int M, int N, int K, EpiArgs E) {
  __shared__ __align__(16) __nv_bfloat16 As[TM][SP];   // [m][k]
  __shared__ __align__(16) __nv_bfloat16 Bs[TN][SP];   // [n][k]
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int g = lane >> 2, t4 = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16(0.f);
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int e = threadIdx.x; e < TM * TK; e += blockDim.x) {
      const int r = e / TK, c = e % TK;
      const int m = m0 + r, k = k0 + c;
      As[r][c] = (m < M && k < K) ? A.p[m * A.sr + k * A.sc] : zero;
      const int n = n0 + r;
      Bs[r][c] = (n < N && k < K) ? B.p[k * B.sr + n * B.sc] : zero;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int ra = wm + 16 * i;
      uint32_t a0 = ld32(&As[ra + g][2 * t4]), a1 = ld32(&As[ra + g + 8][2 * t4]);
      uint32_t a2 = ld32(&As[ra + g][2 * t4 + 8]), a3 = ld32(&As[ra + g + 8][2 * t4 + 8]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int nb = wn + 8 * j;
        uint32_t b0 = ld32(&Bs[nb + g][2 * t4]), b1 = ld32(&Bs[nb + g][2 * t4 + 8]);
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
            "{%0, %1, %2, %3};"
            : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int m = m0 + wm + 16 * i + g + (r >> 1) * 8;
        const int n = n0 + wn + 8 * j + 2 * t4 + (r & 1);
        if (m >= M || n >= N) continue;
        const float v = acc[i][j][r];
        const long o = (long)m * N + n;
        if (E.mode == EPI_FWD_HIDDEN) {
          const float z = v + E.bias[n];
          E.z[o] = z;
          E.act[o] = __float2bfloat16(gelu(z));
        } else if (E.mode == EPI_FWD_OUT) {
          E.z[o] = v + E.bias[n];
        } else if (E.mode == EPI_DX) {
          const float d = v * gelu_grad(E.zprev[o]);
          E.dz32[o] = d;
          E.act[o] = __float2bfloat16(d);
        } else {
          E.z[o] = v;
        }
      }
}

// ---------------------------------------------------------------- small kernels
__global__ void k_set_hyper(float* hyper, float lr, float c1, float c2) {
  hyper[0] = lr;
  hyper[1] = c1;
  hyper[2] = c2;
}

// network input: standardised features, x' = (x - shift) * scale per feature
__global__ void k_inputs(const float* x, const float* shift, const float* scale, __nv_bfloat16* y, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int f = (int)(i % 6);
    y[i] = __float2bfloat16((x[i] - shift[f]) * scale[f]);
  }
}

// network output in the target's units: mu = mu'/ys + y0, log sigma^2 = l' - 2 ln ys
__global__ void k_outputs(const float* z, float y0, float ys, float* out, int B) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    out[2 * b] = z[2 * b] / ys + y0;
    out[2 * b + 1] = z[2 * b + 1] - 2.0f * logf(ys);
  }
}

__global__ void k_to_bf16(const float* x, __nv_bfloat16* y, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    y[i] = __float2bfloat16(x[i]);
}

// Gaussian NLL of the two output heads on the standardised target y' = (y - y0) ys: loss (mean
// over the batch) and dL/d(mu', l').
__global__ void k_nll(const float* out, const float* y, float y0, float ys, int B, float* dz32, __nv_bfloat16* dz16,
                      float* loss) {
  __shared__ float red[256];
  float acc = 0.f;
  for (int b = threadIdx.x; b < B; b += blockDim.x) {
    const float mu = out[2 * b], l = out[2 * b + 1];
    const float r = (y[b] - y0) * ys - mu, w = __expf(-l);
    acc += 0.5f * (r * r * w + l);
    const float dmu = -r * w / B, dl = 0.5f * (1.0f - r * r * w) / B;
    dz32[2 * b] = dmu;
    dz32[2 * b + 1] = dl;
    dz16[2 * b] = __float2bfloat16(dmu);
    dz16[2 * b + 1] = __float2bfloat16(dl);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) *loss = red[0] / B;
}

// db(n) = sum_b dZ(b, n), one thread per output unit, fixed order
__global__ void k_bias_grad(const float* dz, int B, int N, float* db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += dz[(long)b * N + n];
  db[n] = s;
}

// Adam on the FP32 master parameters, then the BF16 copies of the weight matrices.  The step's
// learning rate and bias corrections come from device memory (hyper = {lr, 1 - b1^t, 1 - b2^t}),
// so that a captured training step can be replayed.
__global__ void k_adam(float* p, const float* g, float* m, float* v, long n, const float* hyper, float b1, float b2,
                       float eps) {
  const float lr = hyper[0], c1 = hyper[1], c2 = hyper[2];
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}


// ---------------------------------------------------------------- fused inference on tcgen05
// One CTA (256 threads) per SM, persistent over tiles of 128 rows.  Layer 0 (K = 6) and the
// output layer (N = 2) run on the CUDA cores; the three 256 x 256 layers are single-CTA
// tcgen05.mma (kind::f16, BF16 operands, M = 128, N = 256, K = 16 per instruction) from shared
// memory into an FP32 accumulator of 256 tensor-memory columns.  Operands use the K-major
// no-swizzle canonical layout: element (r, k) of a 256-wide operand at byte
//     (r / 8) * 4096 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// i.e. 8 x 8 core matrices of 128 contiguous bytes, K-adjacent core matrices 128 B apart (the
// descriptor's leading byte offset) and 8-row groups 4096 B apart (its stride byte offset).
// The weights of layers 1-3 are kept in global memory in exactly that image (packed after every
// update) and brought in with one bulk asynchronous copy per layer, overlapping the previous
// layer's epilogue.  The epilogue adds the bias, applies GELU and writes the BF16 activation
// back into the operand buffer; after layer 3 it contracts with the output weights.
namespace tc {

constexpr int THREADS = 512;
constexpr int TILE = 128;
constexpr uint32_t OP_BYTES_A = TILE * 256 * 2;   // 64 KB
constexpr uint32_t OP_BYTES_W = 256 * 256 * 2;    // 128 KB
constexpr uint32_t OFF_A = 0;
constexpr uint32_t OFF_W = OFF_A + OP_BYTES_A;
constexpr uint32_t OFF_W0 = OFF_W + OP_BYTES_W;   // float [256][6]
constexpr uint32_t OFF_B = OFF_W0 + 256 * 6 * 4;  // float [4][256]: b0..b3
constexpr uint32_t OFF_W4 = OFF_B + 4 * 256 * 4;  // float [2][256]
constexpr uint32_t OFF_RED = OFF_W4 + 2 * 256 * 4;  // float [4][128][2]
constexpr uint32_t OFF_MISC = OFF_RED + 4 * TILE * 2 * 4;
constexpr uint32_t SMEM = OFF_MISC + 64;
constexpr long long WAIT_CYCLES = 4000000000LL;   // about two seconds at the maximum clock

// instruction descriptor: D FP32, A and B BF16, both K-major, N = 128 (one column half), M = 128
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((128u >> 3) << 17) | ((128u >> 4) << 24);

__host__ __device__ __forceinline__ uint32_t op_offset(int r, int k) {
  return (uint32_t)((r >> 3) * 4096 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(4096u >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Waits for the phase with the given parity to complete; false after WAIT_CYCLES.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > WAIT_CYCLES) return false;
  }
}

__device__ __forceinline__ void load_weights(uint32_t dst, const void* src, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(OP_BYTES_W) : "memory");
  for (uint32_t c = 0; c < OP_BYTES_W; c += 32768)
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst + c),
                 "l"((const char*)src + c), "r"(32768u), "r"(bar)
                 : "memory");
}

// D[:, 0:128) = A W_half^T over K = 256 (16 instructions); W_half = rows [128 h, 128 h + 128) of W
__device__ __forceinline__ void mma_half(uint32_t tmem_d, uint32_t a_base, uint32_t w_base) {
#pragma unroll
  for (int kk = 0; kk < 16; ++kk) {
    const uint64_t ad = smem_desc(a_base + kk * 256), bd = smem_desc(w_base + kk * 256);
    const uint32_t acc = kk > 0 ? 1u : 0u;
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\ttcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
            tmem_d),
        "l"(ad), "l"(bd), "r"(IDESC), "r"(acc)
        : "memory");
  }
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

__device__ __forceinline__ float round_bf16(float a) { return __bfloat162float(__float2bfloat16(a)); }

// x [B][6] fp32 features; wpack: layers 1-3 in the operand image; wbf: all parameters in BF16
// (W0 and W4 read from it); params: FP32 parameters (biases read from it).  Writes out [B][2]
// = (mu, log sigma^2) in the target's units.  *err is set to 1 if a wait timed out.
// 16 warps: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (its rows) and columns
// [64 (w / 4), + 64).  Each layer's MMAs run as two column halves with their own commits, so
// the warps of half 0 start their epilogue while half 1 is still multiplying; every warp holds
// its BF16 results in registers until both halves are done (all of A feeds both halves).
__global__ void __launch_bounds__(THREADS, 1)
k_mlp_forward(const float* __restrict__ x, int B, const __nv_bfloat16* __restrict__ wpack,
              const __nv_bfloat16* __restrict__ wbf, const float* __restrict__ params, const float* __restrict__ shift,
              const float* __restrict__ scale, float y0, float ys, float* __restrict__ out, int* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  float* sW0 = reinterpret_cast<float*>(sm + OFF_W0);
  float* sB = reinterpret_cast<float*>(sm + OFF_B);
  float* sW4 = reinterpret_cast<float*>(sm + OFF_W4);
  float* sRed = reinterpret_cast<float*>(sm + OFF_RED);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + OFF_MISC);  // [0] weights, [1] MMA half 0, [2] MMA half 1
  uint32_t* sTmem = reinterpret_cast<uint32_t*>(sm + OFF_MISC + 24);
  int* sAbort = reinterpret_cast<int*>(sm + OFF_MISC + 28);
  float* sB4 = reinterpret_cast<float*>(sm + OFF_MISC + 32);
  const int tid = threadIdx.x, warp = tid >> 5;
  const uint32_t a_base = saddr(sm + OFF_A), w_base = saddr(sm + OFF_W);
  const uint32_t barW = saddr(&bars[0]), barM0 = saddr(&bars[1]), barM1 = saddr(&bars[2]);
  const int ntiles = (B + TILE - 1) / TILE;

  // small parameters (BF16 weights as the GEMM path rounds them, FP32 biases)
  constexpr long W0OFF = 0, B0OFF = 6 * 256;
  for (int i = tid; i < 256 * 6; i += THREADS) sW0[i] = __bfloat162float(wbf[W0OFF + i]);
  for (int l = 0; l < 4; ++l) {
    const long bo = (l == 0) ? B0OFF : B0OFF + 256 + (long)(l - 1) * (256 * 256 + 256) + 256 * 256;
    for (int i = tid; i < 256; i += THREADS) sB[l * 256 + i] = params[bo + i];
  }
  const long w4off = B0OFF + 256 + 3L * (256 * 256 + 256);
  for (int i = tid; i < 2 * 256; i += THREADS) sW4[i] = __bfloat162float(wbf[w4off + i]);
  if (tid < 2) sB4[tid] = params[w4off + 2 * 256 + tid];
  if (tid == 0) {
    *sAbort = 0;
    mbar_init(barW, 1);
    mbar_init(barM0, 1);
    mbar_init(barM1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    const uint32_t dst = saddr(sTmem);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(256u) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *sTmem;
  uint32_t phW = 0, phM = 0;
  if (tid == 0 && blockIdx.x < ntiles) load_weights(w_base, wpack, barW);

  const int q = warp & 3, cq = warp >> 2;    // TMEM lane quarter and column quarter of this warp
  const int half = cq >> 1;                  // MMA column half whose commit this warp waits for
  const int erow = 32 * q + (tid & 31);      // epilogue row
  const uint32_t bar_mine = half ? barM1 : barM0;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const bool more = tile + (int)gridDim.x < ntiles;
    // layer 0 on the CUDA cores: row r, columns [64 h, 64 h + 64)
    {
      const int r = tid & (TILE - 1), h = tid >> 7;
      const long row = (long)tile * TILE + r;
      float xin[6];
#pragma unroll
      for (int f = 0; f < 6; ++f) xin[f] = row < B ? round_bf16((x[row * 6 + f] - shift[f]) * scale[f]) : 0.f;
      for (int c0 = 64 * h; c0 < 64 * h + 64; c0 += 8) {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 8; j += 2) {
          float z[2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const float* wr = sW0 + (c0 + j + u) * 6;
            float acc = 0.f;
#pragma unroll
            for (int f = 0; f < 6; ++f) acc = fmaf(xin[f], wr[f], acc);
            z[u] = gelu(acc + sB[c0 + j + u]);
          }
          w[j >> 1] = pack_bf16(z[0], z[1]);
        }
        *reinterpret_cast<uint4*>(sm + OFF_A + op_offset(r, c0)) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    for (int l = 1; l <= 3; ++l) {
      if (tid == 0) {
        if (!mbar_wait(barW, phW)) {
          *sAbort = 1;
        } else {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          mma_half(tmem, a_base, w_base);
          mma_commit(barM0);
          mma_half(tmem + 128, a_base, w_base + 65536);
          mma_commit(barM1);
        }
      }
      phW ^= 1;
      __syncthreads();
      if (*sAbort) break;
      // warp-uniform outcome: tcgen05.ld below is a warp-wide instruction
      bool ok = __all_sync(0xffffffffu, mbar_wait(bar_mine, phM));
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16);
      const float* bias = sB + l * 256;
      uint32_t packed[32];
      float o0 = 0.f, o1 = 0.f;
      if (ok) {
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {
          const int c0 = 64 * cq + 16 * cc;
          float v[16];
          tmem_ld16(trow + c0, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = gelu(v[i] + bias[c0 + i]);
          if (l < 3) {
#pragma unroll
            for (int i = 0; i < 8; ++i) packed[8 * cc + i] = pack_bf16(v[2 * i], v[2 * i + 1]);
          } else {
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const float a = round_bf16(v[i]);
              o0 = fmaf(a, sW4[c0 + i], o0);
              o1 = fmaf(a, sW4[256 + c0 + i], o1);
            }
          }
        }
      }
      // every MMA of the layer is done before the operand buffers are overwritten; the weight
      // buffer is then free for the next layer's (or the next tile's first) weights
      if (half == 0 && l < 3) ok = __all_sync(0xffffffffu, ok && mbar_wait(barM1, phM));
      if (!ok) atomicExch(sAbort, 1);
      phM ^= 1;
      if (tid == 256 && ok && (l < 3 || more))
        load_weights(w_base, wpack + (size_t)(l < 3 ? l : 0) * 256 * 256, barW);
      if (ok && l < 3) {
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) {
          const int c0 = 64 * cq + 8 * cc;
          *reinterpret_cast<uint4*>(sm + OFF_A + op_offset(erow, c0)) =
              make_uint4(packed[4 * cc], packed[4 * cc + 1], packed[4 * cc + 2], packed[4 * cc + 3]);
        }
      }
      if (l == 3) {
        sRed[(cq * TILE + erow) * 2] = o0;
        sRed[(cq * TILE + erow) * 2 + 1] = o1;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      if (*sAbort) break;
    }
    if (*sAbort) break;
    if (tid < TILE) {
      const long row = (long)tile * TILE + tid;
      if (row < B) {
        float z0 = sB4[0], z1 = sB4[1];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          z0 += sRed[(c * TILE + tid) * 2];
          z1 += sRed[(c * TILE + tid) * 2 + 1];
        }
        out[row * 2] = z0 / ys + y0;
        out[row * 2 + 1] = z1 - 2.0f * logf(ys);
      }
    }
  }
  if (*sAbort && tid == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u) : "memory");
}

// Operand image of the weights of layers 1-3 (W[n][k] as the B operand: row n, column k).
__global__ void k_pack_weights(const __nv_bfloat16* __restrict__ wbf, __nv_bfloat16* __restrict__ wpack) {
  const long per = 256L * 256;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < 3 * per; i += (long)gridDim.x * blockDim.x) {
    const int l = (int)(i / per) + 1;
    const int n = (int)((i % per) / 256), k = (int)(i % 256);
    const long woffl = 6 * 256 + 256 + (long)(l - 1) * (256 * 256 + 256);
    wpack[(l - 1) * per + op_offset(n, k) / 2] = wbf[woffl + (long)n * 256 + k];
  }
}

}  // namespace tc
}  // namespace mlp
}  // namespace swf

using namespace swf;
using namespace swf::mlp;

struct swf_mlp {
  int device;
  int max_batch;
  long step;
  float* params;             // FP32 master: per layer W [out][in] then b [out]
  float* grads;
  float* adam_m;
  float* adam_v;
  __nv_bfloat16* wbf;        // BF16 copy of all parameters (same layout)
  __nv_bfloat16* act[NL];    // bf16 input of layer l: [B][DIN[l]]
  float* z[NL];              // fp32 pre-activation of layer l: [B][DOUT[l]]
  float* dz32[NL];           // fp32 dL/dz of layer l
  __nv_bfloat16* dz16[NL];   // bf16 copy
  float* loss;
  float* in_shift;           // [6] feature standardisation
  float* in_scale;           // [6]
  float y0, ys;              // target standardisation
  __nv_bfloat16* wpack;      // layers 1-3 in the tensor-core operand image (inference kernel)
  int* err;                  // set by the inference kernel when a wait timed out
  int nsm;
  cudaStream_t last_stream;
  float* xs;                 // training batch staged for the captured step: [max_batch][6]
  float* ysg;                // [max_batch]
  float* hyper;              // {lr, 1 - b1^t, 1 - b2^t} of the current step
  cudaStream_t cap_stream;   // stream the training step is captured on
  std::map<int, cudaGraphExec_t> train_graphs;  // captured training step per batch size
  std::vector<void*> allocs;
};

namespace {
long woff(int l) {
  long o = 0;
  for (int i = 0; i < l; ++i) o += (long)DIN[i] * DOUT[i] + DOUT[i];
  return o;
}
long boff(int l) { return woff(l) + (long)DIN[l] * DOUT[l]; }

swf_status mlp_alloc(swf_mlp* m, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc failed for the surrogate network");
    return SWF_ENOMEM;
  }
  m->allocs.push_back(*p);
  return SWF_OK;
}

void gemm(const Mat& A, const Mat& B, int M, int N, int K, const EpiArgs& E, cudaStream_t st) {
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  k_gemm<<<grid, 128, 0, st>>>(A, B, M, N, K, E);
}

void refresh_bf16(swf_mlp* m, cudaStream_t st) {
  k_to_bf16<<<128, 256, 0, st>>>(m->params, m->wbf, n_params());
  tc::k_pack_weights<<<192, 256, 0, st>>>(m->wbf, m->wpack);
}

// forward pass on x (fp32 [B][6]); leaves activations for the backward pass; output in z[NL-1]
void forward(swf_mlp* m, const float* x, int B, cudaStream_t st) {
  k_inputs<<<64, 256, 0, st>>>(x, m->in_shift, m->in_scale, m->act[0], (long)B * DIN[0]);
  for (int l = 0; l < NL; ++l) {
    const Mat A = {m->act[l], DIN[l], 1};
    const Mat W = {m->wbf + woff(l), 1, DIN[l]};  // B(k, n) = W[n][k]
    EpiArgs E = {};
    E.mode = l < NL - 1 ? EPI_FWD_HIDDEN : EPI_FWD_OUT;
    E.bias = m->params + boff(l);
    E.z = m->z[l];
    E.act = l < NL - 1 ? m->act[l + 1] : nullptr;
    gemm(A, W, B, DOUT[l], DIN[l], E, st);
  }
}

// backward pass from dz of the output layer; fills m->grads
void backward(swf_mlp* m, int B, cudaStream_t st) {
  for (int l = NL - 1; l >= 0; --l) {
    // dW(n, k) = sum_b dZ(b, n) X(b, k)
    const Mat dZt = {m->dz16[l], 1, DOUT[l]};  // A(n, b) = dZ[b][n]
    const Mat X = {m->act[l], DIN[l], 1};      // B(b, k) = X[b][k]
    EpiArgs E = {};
    E.mode = EPI_DW;
    E.z = m->grads + woff(l);
    gemm(dZt, X, DOUT[l], DIN[l], B, E, st);
    k_bias_grad<<<(DOUT[l] + 127) / 128, 128, 0, st>>>(m->dz32[l], B, DOUT[l], m->grads + boff(l));
    if (l > 0) {
      // dX(b, k) = sum_n dZ(b, n) W(n, k), then times GELU'(z_{l-1})
      const Mat dZ = {m->dz16[l], DOUT[l], 1};
      const Mat W = {m->wbf + woff(l), DIN[l], 1};  // B(n, k) = W[n][k]
      EpiArgs D = {};
      D.mode = EPI_DX;
      D.zprev = m->z[l - 1];
      D.dz32 = m->dz32[l - 1];
      D.act = m->dz16[l - 1];
      gemm(dZ, W, B, DIN[l], DOUT[l], D, st);
    }
  }
}
}  // namespace

extern "C" {

int swf_mlp_param_count(void) { return n_params(); }

swf_status swf_mlp_create(swf_mlp** out, int device, const float* init_params, int max_batch, const float* norm) {
  if (!out || !init_params || !norm || max_batch < 1) { set_error("swf_mlp_create: invalid arguments"); return SWF_EINVAL; }
  if (!(norm[13] > 0.f)) { set_error("swf_mlp_create: target scale must be positive"); return SWF_EINVAL; }
  *out = nullptr;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_status(e, "cudaSetDevice");
  swf_mlp* m = new swf_mlp();
  m->device = device;
  m->max_batch = max_batch;
  m->step = 0;
  const size_t np = n_params();
  swf_status s;
  auto fail = [&](swf_status st) {
    for (void* p : m->allocs) cudaFree(p);
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    delete m;
    return st;
  };
  if ((s = mlp_alloc(m, (void**)&m->params, np * 4)) != SWF_OK) return fail(s);
  if ((s = mlp_alloc(m, (void**)&m->grads, np * 4)) != SWF_OK) return fail(s);
  if ((s = mlp_alloc(m, (void**)&m->adam_m, np * 4)) != SWF_OK) return fail(s);
  if ((s = mlp_alloc(m, (void**)&m->adam_v, np * 4)) != SWF_OK) return fail(s);
  if ((s = mlp_alloc(m, (void**)&m->wbf, np * 2)) != SWF_OK) return fail(s);
  if ((s = mlp_alloc(m, (void**)&m->loss, 4)) != SWF_OK) return fail(s);
  if ((s = mlp_alloc(m, (void**)&m->in_shift, 6 * 4)) != SWF_OK) return fail(s);
  if ((s = mlp_alloc(m, (void**)&m->in_scale, 6 * 4)) != SWF_OK) return fail(s);
  if ((s = mlp_alloc(m, (void**)&m->wpack, (size_t)3 * 256 * 256 * 2)) != SWF_OK) return fail(s);
  if ((s = mlp_alloc(m, (void**)&m->err, sizeof(int))) != SWF_OK) return fail(s);
  if ((s = mlp_alloc(m, (void**)&m->xs, (size_t)max_batch * DIN[0] * 4)) != SWF_OK) return fail(s);
  if ((s = mlp_alloc(m, (void**)&m->ysg, (size_t)max_batch * 4)) != SWF_OK) return fail(s);
  if ((s = mlp_alloc(m, (void**)&m->hyper, 4 * sizeof(float))) != SWF_OK) return fail(s);
  m->cap_stream = nullptr;
  m->last_stream = 0;
  m->nsm = 0;
  e = cudaDeviceGetAttribute(&m->nsm, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess || m->nsm < 1) return fail(cuda_status(e, "SM count"));
  e = cudaFuncSetAttribute(tc::k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc::SMEM);
  if (e != cudaSuccess) return fail(cuda_status(e, "cudaFuncSetAttribute(k_mlp_forward)"));
  e = cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail(cuda_status(e, "capture stream"));
  m->y0 = norm[12];
  m->ys = norm[13];
  for (int l = 0; l < NL; ++l) {
    if ((s = mlp_alloc(m, (void**)&m->act[l], (size_t)max_batch * DIN[l] * 2)) != SWF_OK) return fail(s);
    if ((s = mlp_alloc(m, (void**)&m->z[l], (size_t)max_batch * DOUT[l] * 4)) != SWF_OK) return fail(s);
    if ((s = mlp_alloc(m, (void**)&m->dz32[l], (size_t)max_batch * DOUT[l] * 4)) != SWF_OK) return fail(s);
    if ((s = mlp_alloc(m, (void**)&m->dz16[l], (size_t)max_batch * DOUT[l] * 2)) != SWF_OK) return fail(s);
  }
  e = cudaMemcpy(m->params, init_params, np * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(cuda_status(e, "upload parameters"));
  e = cudaMemcpy(m->in_shift, norm, 6 * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(cuda_status(e, "upload normalisation"));
  e = cudaMemcpy(m->in_scale, norm + 6, 6 * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(cuda_status(e, "upload normalisation"));
  cudaMemset(m->adam_m, 0, np * 4);
  cudaMemset(m->adam_v, 0, np * 4);
  cudaMemset(m->err, 0, sizeof(int));
  refresh_bf16(m, 0);
  e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(cuda_status(e, "surrogate set-up"));
  *out = m;
  return SWF_OK;
}

swf_status swf_mlp_destroy(swf_mlp* m) {
  if (!m) return SWF_OK;
  cudaSetDevice(m->device);
  cudaDeviceSynchronize();
  for (auto& kv : m->train_graphs) cudaGraphExecDestroy(kv.second);
  if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
  for (void* p : m->allocs) cudaFree(p);
  delete m;
  return SWF_OK;
}

swf_status swf_mlp_forward(swf_mlp* m, const float* x_dev, int B, float* out_dev, void* stream) {
  if (!m || !x_dev || !out_dev || B < 1) { set_error("swf_mlp_forward: invalid arguments"); return SWF_EINVAL; }
  cudaSetDevice(m->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int ntiles = (B + tc::TILE - 1) / tc::TILE;
  const int grid = ntiles < m->nsm ? ntiles : m->nsm;
  tc::k_mlp_forward<<<grid, tc::THREADS, tc::SMEM, st>>>(x_dev, B, m->wpack, m->wbf, m->params, m->in_shift,
                                                         m->in_scale, m->y0, m->ys, out_dev, m->err);
  m->last_stream = st;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "surrogate forward");
  return SWF_OK;
}

swf_status swf_mlp_status(swf_mlp* m) {
  if (!m) { set_error("swf_mlp_status: invalid arguments"); return SWF_EINVAL; }
  cudaSetDevice(m->device);
  cudaError_t e = cudaStreamSynchronize(m->last_stream);
  if (e != cudaSuccess) return cuda_status(e, "surrogate status");
  int flag = 0;
  e = cudaMemcpy(&flag, m->err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e, "surrogate status");
  if (flag) {
    set_error("surrogate inference: a tensor-core wait timed out");
    return SWF_ETIMEOUT;
  }
  return SWF_OK;
}

swf_status swf_mlp_gradients(swf_mlp* m, const float* x_dev, const float* y_dev, int B, float* grad_dev,
                             float* loss_dev, void* stream) {
  if (!m || !x_dev || !y_dev || B < 1 || B > m->max_batch) {
    set_error("swf_mlp_gradients: invalid arguments (batch must be in [1, max_batch])");
    return SWF_EINVAL;
  }
  cudaSetDevice(m->device);
  cudaStream_t st = (cudaStream_t)stream;
  forward(m, x_dev, B, st);
  k_nll<<<1, 256, 0, st>>>(m->z[NL - 1], y_dev, m->y0, m->ys, B, m->dz32[NL - 1], m->dz16[NL - 1],
                           loss_dev ? loss_dev : m->loss);
  backward(m, B, st);
  if (grad_dev) {
    cudaError_t e = cudaMemcpyAsync(grad_dev, m->grads, (size_t)n_params() * 4, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_status(e, "copy gradients");
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "surrogate gradients");
  return SWF_OK;
}

// The kernels of one training step on the staged batch (forward, loss, backward, Adam, BF16
// copies and operand image), B rows.
static void record_train_step(swf_mlp* m, int B, cudaStream_t st) {
  forward(m, m->xs, B, st);
  k_nll<<<1, 256, 0, st>>>(m->z[NL - 1], m->ysg, m->y0, m->ys, B, m->dz32[NL - 1], m->dz16[NL - 1], m->loss);
  backward(m, B, st);
  k_adam<<<128, 256, 0, st>>>(m->params, m->grads, m->adam_m, m->adam_v, n_params(), m->hyper, 0.9f, 0.999f, 1e-8f);
  refresh_bf16(m, st);
}

swf_status swf_mlp_train_step(swf_mlp* m, const float* x_dev, const float* y_dev, int B, float lr, float* loss_dev,
                              void* stream) {
  if (!m || !x_dev || !y_dev || B < 1 || B > m->max_batch) {
    set_error("swf_mlp_train_step: invalid arguments (batch must be in [1, max_batch])");
    return SWF_EINVAL;
  }
  cudaSetDevice(m->device);
  cudaStream_t st = (cudaStream_t)stream;
  // the step runs as one CUDA graph per batch size (about 25 kernels, captured once) on the
  // staged batch; the batch, the learning rate and the bias corrections are set before it
  cudaError_t e = cudaMemcpyAsync(m->xs, x_dev, (size_t)B * DIN[0] * 4, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m->ysg, y_dev, (size_t)B * 4, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "stage the training batch");
  m->step += 1;
  const double b1 = 0.9, b2 = 0.999;
  k_set_hyper<<<1, 1, 0, st>>>(m->hyper, lr, (float)(1.0 - std::pow(b1, (double)m->step)),
                               (float)(1.0 - std::pow(b2, (double)m->step)));
  auto it = m->train_graphs.find(B);
  if (it == m->train_graphs.end()) {
    cudaGraphExec_t exec = nullptr;
    e = cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      record_train_step(m, B, m->cap_stream);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(m->cap_stream, &g);
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
      if (g) cudaGraphDestroy(g);
    }
    if (e != cudaSuccess) return cuda_status(e, "capture the training step");
    it = m->train_graphs.emplace(B, exec).first;
  }
  e = cudaGraphLaunch(it->second, st);
  if (e != cudaSuccess) return cuda_status(e, "training step");
  if (loss_dev) {
    e = cudaMemcpyAsync(loss_dev, m->loss, 4, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_status(e, "copy loss");
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "surrogate update");
  return SWF_OK;
}

swf_status swf_mlp_activation(const float* x_dev, int n, float* gelu_dev, float* grad_dev, void* stream) {
  if (!x_dev || !gelu_dev || !grad_dev || n < 0) { set_error("swf_mlp_activation: invalid arguments"); return SWF_EINVAL; }
  if (n == 0) return SWF_OK;
  const int nb = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
  k_gelu_eval<<<nb, 256, 0, (cudaStream_t)stream>>>(x_dev, n, gelu_dev, grad_dev);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "swf_mlp_activation");
  return SWF_OK;
}

swf_status swf_mlp_get_params(swf_mlp* m, float* params_host) {
  if (!m || !params_host) { set_error("swf_mlp_get_params: invalid arguments"); return SWF_EINVAL; }
  cudaSetDevice(m->device);
  cudaError_t e = cudaMemcpy(params_host, m->params, (size_t)n_params() * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e, "download parameters");
  return SWF_OK;
}

}  // extern "C"
