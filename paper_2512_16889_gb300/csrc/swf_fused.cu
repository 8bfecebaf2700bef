// Fused, persistent march of (2+1)D scattered waves on 256 x 256 grids in complex64
// (Sec. II Eq. 6, Sec. II.A: pseudo-spectral derivative, Dormand-Prince in time).
//
// Layout of the work.  With n_z = 1 and no momentum along z, alpha^x, alpha^y, beta and A_0
// never mix the component pairs {0, 3} and {1, 2} (the spin along z is conserved), so each
// instance splits exactly into two independent two-component "sectors".  One thread-block
// cluster of 16 CTAs marches one sector through every step: CTA r owns the rows
// y in [16 r, 16 r + 16) of both components.  Per right-hand-side evaluation:
//   1. stage combine  Y = y + h sum_j a_ij k_j   (y in shared memory, k_j in the cluster's
//      global slot, which stays resident in L2), local term Z = -i V (Y + psi_b) to a global
//      stash, forward x-FFT of the rows in shared memory;
//   2. cluster barrier; each CTA pulls its 16 columns of every CTA's rows through distributed
//      shared memory (the transpose), forward y-FFT, -i H0(kappa)/N per mode, inverse y-FFT;
//   3. cluster barrier; each CTA pulls its rows back, inverse x-FFT, k_i = (that) + Z.
// Two shared buffers (rows, columns) make each transpose a single pull after one barrier.
// The 256-point FFTs are two radix-16 passes over lines padded by one element per 16 (and one
// more per line) so that the passes and the transposes are free of bank conflicts.
// That is `k_fused`.  The default kernel, `k_fused3` (further below), does the same arithmetic but
// has the bulk-copy engine push the transposes while its threads compute, and `k_fused2` runs two
// smaller CTAs per SM.
#include <cooperative_groups.h>

#include <cstdio>
#include <cstring>

#include "swf_internal.h"

namespace cg = cooperative_groups;

namespace swf {

namespace fused {

constexpr int NT = 512;         // threads per CTA
constexpr int CL = 16;          // CTAs per cluster
constexpr int NX = 256;         // points along x
constexpr int NY = 256;         // points along y
constexpr int RB = NY / CL;     // rows per CTA
constexpr int CB = NX / CL;     // columns per CTA
constexpr int LD = 273;         // padded line stride (complex): 256 + 16 + 1
constexpr int NSL = 2 * RB * NX;  // complex values in one CTA slab (both components)

__host__ __device__ constexpr int pidx(int i) { return i + (i >> 4); }

struct Sector {      // one marched two-component field
  int inst;          // instance index (output slot)
  int c0, c1;        // components of the 4-spinor
  int sigma;         // +1 for {0, 3}, -1 for {1, 2} (sign of the y coupling)
};

struct Args {
  const FieldDesc* fd;     // per instance
  const Sector* sec;       // per sector
  int n_sec;
  float2* slots;           // per cluster, arrays of 2 NX NY complex: k_4..k_6 and the low part of y
                           // (k_fused, k_fused3), or k_2..k_6, y and its low part (k_fused2)
  float2* psi_out;         // [inst][4][NY][NX] complex64
  double Lx, Ly, t_out, h;
  int n_steps;
  const float4* ttab;      // per instance [n_steps][7]: field time factor, background time phase (re, im)
  int* status;             // k_fused3: set to 1 when a receive wait ran out (may be null)
  int drop;                // k_fused3 diagnostic: nonzero = no CTA copies, so every receive wait runs out
};

// shared-memory map (bytes)
constexpr int OFF_WA = 0;                                   // [2][RB][LD] complex
constexpr int OFF_WB = OFF_WA + 2 * RB * LD * 8;            // [2][CB][LD] complex
constexpr int OFF_Y = OFF_WB + 2 * CB * LD * 8;             // [2][RB][NX] complex (state y)
constexpr int OFF_TW = OFF_Y + NSL * 8;                     // [256] complex twiddles
constexpr int OFF_EX = OFF_TW + 256 * 8;                    // [NX] complex  exp(i p_x x)
constexpr int OFF_GX = OFF_EX + NX * 8;                     // [NX] float    field x factor
constexpr int OFF_EY = OFF_GX + NX * 4;                     // [RB] complex
constexpr int OFF_GY = OFF_EY + RB * 8;                     // [RB] float
constexpr int OFF_KX = OFF_GY + RB * 4;                     // [NX] float   kappa_x of the mode
constexpr int OFF_KY = OFF_KX + NX * 4;                     // [NY] float   sigma kappa_y of the mode
constexpr int OFF_MISC = OFF_KY + NY * 4;                   // per-stage scalars
constexpr int SMEM = OFF_MISC + 7 * RB * 4 + 7 * 8 + 16 + 64 + 16;

__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// Complex products with every rounding fixed (one product, then one fused multiply-add per
// part), so that the fused kernels, however the compiler schedules them, give the same bits.
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, -__fmul_rn(a.y, b.y)), __fmaf_rn(a.x, b.y, __fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
  return make_float2(__fmaf_rn(a.x, b.x, __fmul_rn(a.y, b.y)), __fmaf_rn(a.y, b.x, -__fmul_rn(a.x, b.y)));
}
__device__ __forceinline__ float2 scl(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__device__ __forceinline__ float2 fma2(float s, float2 a, float2 c) {
  return make_float2(fmaf(s, a.x, c.x), fmaf(s, a.y, c.y));
}
// multiply by -i (forward) or +i (inverse)
template <bool INV> __device__ __forceinline__ float2 rot(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// y += c k on both complex halves of a float4 (two-lane FP32 fused multiply-adds)
__device__ __forceinline__ void fma4(float2 c, const float4& k, float4& y) {
  const float2 lo = __ffma2_rn(c, make_float2(k.x, k.y), make_float2(y.x, y.y));
  const float2 hi = __ffma2_rn(c, make_float2(k.z, k.w), make_float2(y.z, y.w));
  y = make_float4(lo.x, lo.y, hi.x, hi.y);
}

// (hi, lo) + s in float-float arithmetic (Knuth's two-sum, then a fast renormalisation):
// on return hi is the new rounded state, lo its rounding error; s is overwritten with hi.
__device__ __forceinline__ void ff_add(float hi, float& lo, float& s) {
  const float t = hi + s;
  const float bp = t - hi;
  const float e = (hi - (t - bp)) + (s - bp);
  const float l = lo + e;
  const float nh = t + l;
  lo = l - (nh - t);
  s = nh;
}

// ---- tensor memory (TMEM) as per-thread storage: 32-bit lanes x columns, warp w reaches lanes
// 32 (w % 4) .. 32 (w % 4) + 31; the 32x32b shape gives each thread its own lane.
__device__ __forceinline__ void tmem_alloc(uint32_t* smem_dst, uint32_t ncols) {
  const uint32_t dst = (uint32_t)__cvta_generic_to_shared(smem_dst);
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// 8 consecutive columns of this thread's lane -> two float4
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float4& a, float4& b) {
  uint32_t r0, r1, r2, r3, r4, r5, r6, r7;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3), "=r"(r4), "=r"(r5), "=r"(r6), "=r"(r7)
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  a = make_float4(__uint_as_float(r0), __uint_as_float(r1), __uint_as_float(r2), __uint_as_float(r3));
  b = make_float4(__uint_as_float(r4), __uint_as_float(r5), __uint_as_float(r6), __uint_as_float(r7));
}
// 16 consecutive columns of this thread's lane -> four float4
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float4& a, float4& b, float4& c, float4& d) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  a = make_float4(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]), __uint_as_float(r[3]));
  b = make_float4(__uint_as_float(r[4]), __uint_as_float(r[5]), __uint_as_float(r[6]), __uint_as_float(r[7]));
  c = make_float4(__uint_as_float(r[8]), __uint_as_float(r[9]), __uint_as_float(r[10]), __uint_as_float(r[11]));
  d = make_float4(__uint_as_float(r[12]), __uint_as_float(r[13]), __uint_as_float(r[14]), __uint_as_float(r[15]));
}
// 8 columns without waiting (pair with tmem_wait_ld before the registers are read)
__device__ __forceinline__ void tmem_ld8_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const float4& a, const float4& b) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"r"(taddr),
               "r"(__float_as_uint(a.x)), "r"(__float_as_uint(a.y)), "r"(__float_as_uint(a.z)), "r"(__float_as_uint(a.w)),
               "r"(__float_as_uint(b.x)), "r"(__float_as_uint(b.y)), "r"(__float_as_uint(b.z)), "r"(__float_as_uint(b.w))
               : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 4-point DFT on packed pairs: each complex add or subtract is one two-lane FP32 instruction
// (add.f32x2 / fma.f32x2 with an exact +-1 factor, so every result is the same single rounding
// as the scalar form); the +-i rotation is a lane swap with the sign folded into the factor.
template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 t0 = __fadd2_rn(a0, a2);
  const float2 t1 = __ffma2_rn(a2, m1, a0);
  const float2 t2 = __fadd2_rn(a1, a3);
  const float2 d = __ffma2_rn(a3, m1, a1);
  const float2 sw = make_float2(d.y, d.x);
  // rot(d) = -i d = (d.y, -d.x) forward, +i d = (-d.y, d.x) inverse
  const float2 sp = INV ? make_float2(-1.f, 1.f) : make_float2(1.f, -1.f);
  const float2 sn = INV ? make_float2(1.f, -1.f) : make_float2(-1.f, 1.f);
  a0 = __fadd2_rn(t0, t2);
  a2 = __ffma2_rn(t2, m1, t0);
  a1 = __ffma2_rn(sw, sp, t1);
  a3 = __ffma2_rn(sw, sn, t1);
}

// 16-point DFT in registers, natural order in and out (4 x 4 with the W16 twiddles).
template <bool INV>
__device__ __forceinline__ void dft16(float2* a) {
  // stage 1: DFT4 over n1 for each n2 (index n = 4 n1 + n2), result b[k1][n2] at a[4 k1 + n2]
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4<INV>(a[n2], a[4 + n2], a[8 + n2], a[12 + n2]);
  // twiddles W16^{n2 k1}
  const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, h2 = 0.70710678118654752440f;
  const float sg = INV ? 1.f : -1.f;  // imaginary sign of W16^m = cos - i sin (forward)
  // k1 = 1: m = n2
  a[5] = cmul(a[5], make_float2(c1, sg * s1));
  a[6] = cmul(a[6], make_float2(h2, sg * h2));
  a[7] = cmul(a[7], make_float2(s1, sg * c1));
  // k1 = 2: m = 2 n2
  a[9] = cmul(a[9], make_float2(h2, sg * h2));
  a[10] = rot<INV>(a[10]);
  a[11] = cmul(a[11], make_float2(-h2, sg * h2));
  // k1 = 3: m = 3 n2
  a[13] = cmul(a[13], make_float2(s1, sg * c1));
  a[14] = cmul(a[14], make_float2(-h2, sg * h2));
  a[15] = cmul(a[15], make_float2(-c1, -sg * s1));
  // stage 2: DFT4 over n2 for each k1; X[k1 + 4 k2] = result k2
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4<INV>(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
  // a[4 k1 + k2] holds X[k1 + 4 k2]: transpose the 4x4 index
  float2 t;
  t = a[1]; a[1] = a[4]; a[4] = t;
  t = a[2]; a[2] = a[8]; a[8] = t;
  t = a[3]; a[3] = a[12]; a[12] = t;
  t = a[6]; a[6] = a[9]; a[9] = t;
  t = a[7]; a[7] = a[13]; a[13] = t;
  t = a[11]; a[11] = a[14]; a[14] = t;
}

// In-place 256-point FFT of 32 padded lines (stride LD) with 512 threads: thread t works on
// line t/16, index j = t%16.  Pass 1 combines x[16 n1 + j] over n1 (reads and writes the same
// addresses); pass 2 combines the 16 values of one row of the 16 x 16 decomposition.
template <bool INV>
__device__ __forceinline__ void fft256_lines(float2* buf, const float2* tw) {
  const int l = threadIdx.x >> 4, j = threadIdx.x & 15;
  float2* line = buf + l * LD;
  float2 a[16];
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1) a[n1] = line[17 * n1 + j];
  dft16<INV>(a);
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) {
    const float2 w = tw[(j * k1) & 255];
    a[k1] = INV ? cmulc(a[k1], w) : cmul(a[k1], w);
  }
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) line[17 * k1 + j] = a[k1];
  __syncthreads();
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) a[n2] = line[17 * j + n2];
  dft16<INV>(a);
  __syncthreads();
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) line[j + 17 * k2] = a[k2];
  __syncthreads();
}

__device__ __forceinline__ double time_factor(const FieldDesc& F, double t, double y) {
  switch (F.kind) {
    case SWF_FIELD_SAUTER_GAUSS: {
      const double c = cosh(F.prm[1] * t);
      return (F.prm[0] / F.prm[1]) / (c * c);
    }
    case SWF_FIELD_PULSE_GAUSS: {
      const double u = t - y;
      return F.prm[0] * sin(F.prm[1] * u) * exp(-u * u / (F.prm[2] * F.prm[2]));
    }
    case SWF_FIELD_SINGLE_E:
    case SWF_FIELD_DOUBLE_E: {
      const double a = F.prm[1] * t;
      return exp(-a * a);
    }
    default:
      return 0.0;
  }
}

__device__ __forceinline__ double single_e_x(const FieldDesc& F, double x) {
  const double kx = F.prm[2];
  return -(F.prm[0] / kx) * sin(kx * x) * exp(-(kx * x) * (kx * x));
}

__device__ double axis_factor(const FieldDesc& F, int axis, double xc) {
  switch (F.kind) {
    case SWF_FIELD_SAUTER_GAUSS: {
      const double lam = F.prm[2];
      return lam > 0.0 ? exp(-xc * xc / (lam * lam)) : 1.0;
    }
    case SWF_FIELD_PULSE_GAUSS:
      if (axis == 0) return exp(-xc * xc / (F.prm[3] * F.prm[3]));
      return F.prm[4] > 0.0 ? exp(-xc * xc / (F.prm[4] * F.prm[4])) : 1.0;
    case SWF_FIELD_SINGLE_E:
    case SWF_FIELD_DOUBLE_E:
      if (axis == 0)
        return F.kind == SWF_FIELD_SINGLE_E ? single_e_x(F, xc)
                                            : single_e_x(F, xc + F.prm[5]) + single_e_x(F, xc - F.prm[5]);
      return exp(-(F.prm[3] * xc) * (F.prm[3] * xc));
    default:
      return 0.0;
  }
}

// Time factors of every stage of every step, computed once in FP64 by all SMs in parallel
// (FP64 is scarce on this GPU, so the march itself only reads the rounded table).  Fields
// whose time factor depends on y (the travelling pulse) are not tabulated.
__global__ void k_time_table(const FieldDesc* fd, int n_inst, int n_steps, double t_out, double h, float4* tab) {
  const double DPc[7] = {0.0, 0.2, 0.3, 0.8, 8.0 / 9.0, 1.0, 1.0};
  const size_t total = (size_t)n_inst * n_steps * 7;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int inst = (int)(i / ((size_t)n_steps * 7));
    const int rem = (int)(i % ((size_t)n_steps * 7));
    const int step = rem / 7, st = rem % 7;
    const FieldDesc& F = fd[inst];
    const double t = t_out + step * h + DPc[st] * h;
    double sn, cs;
    sincos(F.tsign * F.e0 * t, &sn, &cs);
    tab[i] = make_float4((float)time_factor(F, t, 0.0), (float)cs, (float)sn, 0.f);
  }
}

// -i H0(kappa)/N of one mode of a sector, (a, b) -> (o0, o1): [[1, kx - i ky], [kx + i ky, -1]]
// (a, b), times -i/N, with every fused multiply-add rounded once in this order, so that every
// fused kernel gives the same bits.
__device__ __forceinline__ void h0_pair(float2 a, float2 b, float kx, float ky, float inv_n, float2& o0,
                                        float2& o1) {
  const float2 h0 = make_float2(__fmaf_rn(ky, b.y, __fmaf_rn(kx, b.x, a.x)), __fmaf_rn(-ky, b.x, __fmaf_rn(kx, b.y, a.y)));
  const float2 h1 = make_float2(__fmaf_rn(-ky, a.y, __fmaf_rn(kx, a.x, -b.x)), __fmaf_rn(ky, a.x, __fmaf_rn(kx, a.y, -b.y)));
  o0 = scl(inv_n, rot<false>(h0));
  o1 = scl(inv_n, rot<false>(h1));
}

// V (phi0, phi1) for the sector (components c0, c1) with the one non-zero A_mu = a.
__device__ __forceinline__ void sector_v(int acomp, int sigma, float a, float2 p0, float2 p1, float2& o0, float2& o1) {
  if (acomp == 0) {
    o0 = scl(a, p0);
    o1 = scl(a, p1);
  } else if (acomp == 1) {  // alpha^x swaps the pair
    o0 = scl(a, p1);
    o1 = scl(a, p0);
  } else if (acomp == 2) {  // alpha^y: [[0, -i sigma], [i sigma, 0]]
    const float sa = sigma * a;
    o0 = make_float2(sa * p1.y, -sa * p1.x);
    o1 = make_float2(-sa * p0.y, sa * p0.x);
  } else {
    o0 = make_float2(0.f, 0.f);
    o1 = o0;
  }
}

__global__ void __launch_bounds__(NT, 1) k_fused(Args A) {
  extern __shared__ __align__(16) unsigned char sm[];
  float2* WA = reinterpret_cast<float2*>(sm + OFF_WA);
  float2* WB = reinterpret_cast<float2*>(sm + OFF_WB);
  float2* Ys = reinterpret_cast<float2*>(sm + OFF_Y);
  float2* tw = reinterpret_cast<float2*>(sm + OFF_TW);
  float2* ex = reinterpret_cast<float2*>(sm + OFF_EX);
  float* gx = reinterpret_cast<float*>(sm + OFF_GX);
  float2* ey = reinterpret_cast<float2*>(sm + OFF_EY);
  float* gy = reinterpret_cast<float*>(sm + OFF_GY);
  float* kxt = reinterpret_cast<float*>(sm + OFF_KX);
  float* kyt = reinterpret_cast<float*>(sm + OFF_KY);
  float* s_ft = reinterpret_cast<float*>(sm + OFF_MISC);                     // [7][RB] field time factor
  float2* s_tf = reinterpret_cast<float2*>(sm + OFF_MISC + 7 * RB * 4);      // [7] background time phase
  float2* s_w = reinterpret_cast<float2*>(sm + OFF_MISC + 7 * RB * 4 + 56);  // sector spinor [2]
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + OFF_MISC + 7 * RB * 4 + 72);

  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int cid = blockIdx.x / CL;
  const int ncl = gridDim.x / CL;
  const int tid = threadIdx.x;
  const int row0 = rank * RB;
  const size_t plane = (size_t)NX * NY;
  // global slot of the cluster: k_4, k_5, k_6 and the low part of y; k_1 (= k_7 of the previous
  // step), k_2, k_3 and the local-term stash live in tensor memory, 128 columns each
  float2* slot = A.slots + (size_t)cid * 4 * 2 * plane;
  const int warp = tid >> 5;
  if (warp == 0) {
    tmem_alloc(s_tmem, 512);
    tmem_relinquish();
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *s_tmem;
  // this thread's 32 columns in each slab: lane quarter warp % 4, column group warp / 4
  const uint32_t tme = tbase + (((uint32_t)(32 * (warp & 3))) << 16) + 32 * (warp >> 2);

  for (int m = tid; m < 256; m += NT) {
    double s, c;
    sincospi(-2.0 * m / 256.0, &s, &c);
    tw[m] = make_float2((float)c, (float)s);
  }
  const double dxx = A.Lx / NX, dyy = A.Ly / NY;
  const float inv_n = 1.0f / (float)(NX * NY);
  // Dormand-Prince tableau (Dormand & Prince 1980), first same as last
  const double DPc[7] = {0.0, 0.2, 0.3, 0.8, 8.0 / 9.0, 1.0, 1.0};
  const double DPa[7][6] = {{0, 0, 0, 0, 0, 0},
                            {0.2, 0, 0, 0, 0, 0},
                            {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
                            {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
                            {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
                            {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
                            {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};

  for (int si = cid; si < A.n_sec; si += ncl) {
    const Sector S = A.sec[si];
    const FieldDesc& F = A.fd[S.inst];
    // per-sector tables (FP64, rounded once)
    for (int i = tid; i < NX; i += NT) {
      const double xc = -0.5 * A.Lx + i * dxx;
      gx[i] = (float)axis_factor(F, 0, xc);
      double s, c;
      sincos(F.pmom[0] * xc, &s, &c);
      ex[i] = make_float2((float)c, (float)s);
    }
    if (tid < RB) {
      const double yc = -0.5 * A.Ly + (row0 + tid) * dyy;
      gy[tid] = (float)axis_factor(F, 1, yc);
      double s, c;
      sincos(F.pmom[1] * yc, &s, &c);
      ey[tid] = make_float2((float)c, (float)s);
    }
    for (int i = tid; i < NX; i += NT) kxt[i] = (float)(6.283185307179586476925286766559 * (i < NX / 2 ? i : i - NX) / A.Lx);
    for (int i = tid; i < NY; i += NT)
      kyt[i] = (float)(S.sigma * 6.283185307179586476925286766559 * (i < NY / 2 ? i : i - NY) / A.Ly);
    if (tid < 2) {
      const int c = tid == 0 ? S.c0 : S.c1;
      s_w[tid] = make_float2((float)F.w[2 * c], (float)F.w[2 * c + 1]);
    }
    for (int i = tid; i < NSL; i += NT) Ys[i] = make_float2(0.f, 0.f);
    for (int i = tid; i < NSL; i += NT) {
      const int comp = i / (RB * NX), rem = i % (RB * NX);
      __stcg(slot + (size_t)3 * 2 * plane + comp * plane + (size_t)row0 * NX + rem, make_float2(0.f, 0.f));
    }
    __syncthreads();

    // evaluations: e = 0 is k_1 = f(t_out, 0); then 6 per step
    const int n_eval = 1 + 6 * A.n_steps;
    for (int ev = 0; ev < n_eval; ++ev) {
      const int step = ev == 0 ? 0 : (ev - 1) / 6;
      const int stage = ev == 0 ? 0 : 1 + (ev - 1) % 6;  // 0..6 (stage index i)
      // time factors of every stage of this step at once (FP64, rounded once): one FP64
      // latency per step instead of one per evaluation
      if (ev == 0 || stage == 1) {
        const int st0 = ev == 0 ? 0 : 1, nst = ev == 0 ? 1 : 6;
        if (F.kind == SWF_FIELD_PULSE_GAUSS) {
          if (tid < nst * RB) {
            const int si2 = st0 + tid / RB, r = tid % RB;
            const double ts = A.t_out + step * A.h + DPc[si2] * A.h;
            const double yc = -0.5 * A.Ly + (row0 + r) * dyy;
            s_ft[si2 * RB + r] = (float)time_factor(F, ts, yc);
          } else if (tid >= 128 && tid < 128 + nst) {
            const int si2 = st0 + tid - 128;
            const double ts = A.t_out + step * A.h + DPc[si2] * A.h;
            double s, c;
            sincos(F.tsign * F.e0 * ts, &s, &c);
            s_tf[si2] = make_float2((float)c, (float)s);
          }
        } else if (tid < nst * RB) {
          const int si2 = st0 + tid / RB, r = tid % RB;
          const float4 e = __ldg(A.ttab + ((size_t)S.inst * A.n_steps + step) * 7 + si2);
          s_ft[si2 * RB + r] = e.x;
          if (r == 0) s_tf[si2] = make_float2(e.y, e.z);
        }
        __syncthreads();
      }
      // ---- 1. stage combine, local term, rows into WA
      float coef[6];
      const float2* kin[6];
      int nterm = 0;
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        coef[j] = 0.f;
        kin[j] = slot;
      }
      // k_1, k_2, k_3 from tensor memory (coefficients ct[]), k_4 .. k_6 from the global slot
      float ct[3];
#pragma unroll
      for (int j = 0; j < 3; ++j) ct[j] = (j < stage) ? (float)(A.h * DPa[stage][j]) : 0.f;
      const int ntm = stage < 3 ? stage : 3;
#pragma unroll
      for (int j = 3; j < 6; ++j) {
        if (j < stage && DPa[stage][j] != 0.0) {
#pragma unroll
          for (int q = 0; q < 6; ++q)
            if (q == nterm) {
              coef[q] = (float)(A.h * DPa[stage][j]);
              kin[q] = slot + (size_t)(j - 3) * 2 * plane;
            }
          ++nterm;
        }
      }
      // output: stages 0 and 6 (k_1, k_7) -> slab 0, stages 1, 2 -> slabs 1, 2, stages 3..5 -> global
      const int oslab = stage == 0 || stage == 6 ? 0 : (stage <= 2 ? stage : -1);
      float2* kout = slot + (size_t)(stage >= 3 && stage <= 5 ? stage - 3 : 0) * 2 * plane;
      const float2 tf = s_tf[stage];
      const float* ftr = s_ft + stage * RB;
      float2* ylo = slot + (size_t)3 * 2 * plane;
      const float2 w0 = s_w[0], w1 = s_w[1];
#pragma unroll 2
      for (int m = 0; m < 4; ++m) {
        const int sp = tid + NT * m;   // site pair in the slab: 16 rows x 128 pairs
        const int r = sp >> 7;
        const int x = (sp & 127) * 2;
        const size_t g0 = (size_t)(row0 + r) * NX + x;
        const float4 yh0 = *reinterpret_cast<const float4*>(Ys + r * NX + x);
        const float4 yh1 = *reinterpret_cast<const float4*>(Ys + RB * NX + r * NX + x);
        // the last stage accumulates h sum_j b_j k_j separately and adds it to (y, y_low)
        // in float-float arithmetic; other stages form Y from y directly
        const bool last = stage == 6;
        float4 y0 = last ? make_float4(0.f, 0.f, 0.f, 0.f) : yh0;
        float4 y1 = last ? make_float4(0.f, 0.f, 0.f, 0.f) : yh1;
        if (ntm > 0) {
          uint32_t tr[3][8];
#pragma unroll
          for (int j = 0; j < 3; ++j)
            if (j < ntm) tmem_ld8_nowait(tme + 128 * j + 8 * m, tr[j]);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            if (j < ntm) {
              const float2 c = make_float2(ct[j], ct[j]);
              fma4(c, make_float4(__uint_as_float(tr[j][0]), __uint_as_float(tr[j][1]), __uint_as_float(tr[j][2]),
                                  __uint_as_float(tr[j][3])), y0);
              fma4(c, make_float4(__uint_as_float(tr[j][4]), __uint_as_float(tr[j][5]), __uint_as_float(tr[j][6]),
                                  __uint_as_float(tr[j][7])), y1);
            }
          }
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          if (q < nterm) {
            const float4 k0 = __ldcg(reinterpret_cast<const float4*>(kin[q] + g0));
            const float4 k1 = __ldcg(reinterpret_cast<const float4*>(kin[q] + plane + g0));
            const float2 c = make_float2(coef[q], coef[q]);
            fma4(c, k0, y0);
            fma4(c, k1, y1);
          }
        }
        if (last) {
          float4 l0 = __ldcg(reinterpret_cast<const float4*>(ylo + g0));
          float4 l1 = __ldcg(reinterpret_cast<const float4*>(ylo + plane + g0));
          ff_add(yh0.x, l0.x, y0.x); ff_add(yh0.y, l0.y, y0.y); ff_add(yh0.z, l0.z, y0.z); ff_add(yh0.w, l0.w, y0.w);
          ff_add(yh1.x, l1.x, y1.x); ff_add(yh1.y, l1.y, y1.y); ff_add(yh1.z, l1.z, y1.z); ff_add(yh1.w, l1.w, y1.w);
          __stcg(reinterpret_cast<float4*>(ylo + g0), l0);
          __stcg(reinterpret_cast<float4*>(ylo + plane + g0), l1);
          *reinterpret_cast<float4*>(Ys + r * NX + x) = y0;
          *reinterpret_cast<float4*>(Ys + RB * NX + r * NX + x) = y1;
        }
        // rows into WA (padded)
        float2* wa0 = WA + r * LD + pidx(x);
        float2* wa1 = WA + (RB + r) * LD + pidx(x);
        wa0[0] = make_float2(y0.x, y0.y);
        wa0[1] = make_float2(y0.z, y0.w);
        wa1[0] = make_float2(y1.x, y1.y);
        wa1[1] = make_float2(y1.z, y1.w);
        // local term Z = -i V (Y + psi_b) on the two sites
        const float ft = ftr[r];
        const float2 phy = cmul(tf, ey[r]);
        float4 z0, z1;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float2 ph = cmul(phy, ex[x + e]);
          const float a = ft * gy[r] * gx[x + e];
          const float2 p0 = (e ? make_float2(y0.z, y0.w) : make_float2(y0.x, y0.y)) + cmul(w0, ph);
          const float2 p1 = (e ? make_float2(y1.z, y1.w) : make_float2(y1.x, y1.y)) + cmul(w1, ph);
          float2 v0, v1;
          sector_v(F.acomp, S.sigma, a, p0, p1, v0, v1);
          v0 = rot<false>(v0);
          v1 = rot<false>(v1);
          if (e) { z0.z = v0.x; z0.w = v0.y; z1.z = v1.x; z1.w = v1.y; }
          else { z0.x = v0.x; z0.y = v0.y; z1.x = v1.x; z1.y = v1.y; }
        }
        tmem_st8(tme + 128 * 3 + 8 * m, z0, z1);
      }
      tmem_wait_st();
      __syncthreads();
      fft256_lines<false>(WA, tw);
      // ---- 2. transpose rows -> columns through distributed shared memory
      cluster.sync();
      {
        const int comp = tid >> 8, r = (tid >> 4) & 15, col = tid & 15;
#pragma unroll
        for (int i = 0; i < CL; ++i) {
          const int s = (rank + i) & (CL - 1);  // rotated order: no source CTA is read by all at once
          const float2* src = cluster.map_shared_rank(WA, s);
          WB[(comp * CB + col) * LD + pidx(s * RB + r)] = src[(comp * RB + r) * LD + pidx(rank * CB + col)];
        }
      }
      __syncthreads();
      fft256_lines<false>(WB, tw);
      // -i H0(kappa)/N per mode of the sector
      {
#pragma unroll 2
        for (int m = tid; m < CB * NY; m += NT) {
          const int col = m >> 8, iy = m & 255;
          const float kx = kxt[rank * CB + col];
          const float ky = kyt[iy];
          float2* pa = WB + col * LD + pidx(iy);
          float2* pb = WB + (CB + col) * LD + pidx(iy);
          h0_pair(*pa, *pb, kx, ky, inv_n, *pa, *pb);
        }
      }
      __syncthreads();
      fft256_lines<true>(WB, tw);
      // ---- 3. transpose columns -> rows, inverse x-FFT, output
      cluster.sync();
      {
        const int comp = tid >> 8, col = (tid >> 4) & 15, r = tid & 15;
#pragma unroll
        for (int i = 0; i < CL; ++i) {
          const int s = (rank + i) & (CL - 1);
          const float2* src = cluster.map_shared_rank(WB, s);
          WA[(comp * RB + r) * LD + pidx(s * CB + col)] = src[(comp * CB + col) * LD + pidx(rank * RB + r)];
        }
      }
      __syncthreads();
      fft256_lines<true>(WA, tw);
#pragma unroll 4
      for (int m = 0; m < 4; ++m) {
        const int sp = tid + NT * m;
        const int r = sp >> 7;
        const int x = (sp & 127) * 2;
        const size_t g0 = (size_t)(row0 + r) * NX + x;
        float4 z0, z1;
        tmem_ld8(tme + 128 * 3 + 8 * m, z0, z1);
        const float2* wa0 = WA + r * LD + pidx(x);
        const float2* wa1 = WA + (RB + r) * LD + pidx(x);
        const float4 o0 = make_float4(wa0[0].x + z0.x, wa0[0].y + z0.y, wa0[1].x + z0.z, wa0[1].y + z0.w);
        const float4 o1 = make_float4(wa1[0].x + z1.x, wa1[0].y + z1.y, wa1[1].x + z1.z, wa1[1].y + z1.w);
        if (oslab >= 0) {
          tmem_st8(tme + 128 * oslab + 8 * m, o0, o1);
        } else {
          __stcg(reinterpret_cast<float4*>(kout + g0), o0);
          __stcg(reinterpret_cast<float4*>(kout + plane + g0), o1);
        }
      }
      tmem_wait_st();
      __syncthreads();
    }
    // psi(t_in) of the sector into the 4-component output
    float2* out0 = A.psi_out + ((size_t)S.inst * 4 + S.c0) * plane + (size_t)row0 * NX;
    float2* out1 = A.psi_out + ((size_t)S.inst * 4 + S.c1) * plane + (size_t)row0 * NX;
    for (int i = tid; i < RB * NX; i += NT) {
      out0[i] = Ys[i];
      out1[i] = Ys[RB * NX + i];
    }
    __syncthreads();
  }
  // no CTA may exit while another CTA of the cluster can still read its shared memory
  cluster.sync();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, 512);
}


// ------------------------------------------------------------------ two CTAs per SM variant
// 256 threads and one shared buffer per CTA (about 76 KB), so that two CTAs (of two clusters)
// share an SM and hide each other's barrier and memory latency.  y and its low part move to
// the cluster's global slot; each transpose pulls into registers, waits for the whole cluster,
// and then overwrites the buffer in place (two cluster barriers per transpose).
namespace v2 {
constexpr int NT2 = 256;
constexpr int OFF_W = 0;                            // [2][16][LD] complex
constexpr int OFF_TW2 = OFF_W + 2 * 16 * LD * 8;
constexpr int OFF_EX2 = OFF_TW2 + 256 * 8;
constexpr int OFF_GX2 = OFF_EX2 + NX * 8;
constexpr int OFF_EY2 = OFF_GX2 + NX * 4;
constexpr int OFF_GY2 = OFF_EY2 + RB * 8;
constexpr int OFF_KX2 = OFF_GY2 + RB * 4;
constexpr int OFF_KY2 = OFF_KX2 + NX * 4;
constexpr int OFF_MISC2 = OFF_KY2 + NY * 4;
constexpr int SMEM2 = OFF_MISC2 + 7 * RB * 4 + 7 * 8 + 16 + 64;
}  // namespace v2

// two lines per thread: lines t/16 and t/16 + 16
template <bool INV>
__device__ __forceinline__ void fft256_lines2(float2* buf, const float2* tw) {
  const int l = threadIdx.x >> 4, j = threadIdx.x & 15;
  float2* la = buf + l * LD;
  float2* lb = buf + (l + 16) * LD;
  float2 a[16], b[16];
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1) { a[n1] = la[17 * n1 + j]; b[n1] = lb[17 * n1 + j]; }
  dft16<INV>(a);
  dft16<INV>(b);
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) {
    const float2 w = tw[(j * k1) & 255];
    a[k1] = INV ? cmulc(a[k1], w) : cmul(a[k1], w);
    b[k1] = INV ? cmulc(b[k1], w) : cmul(b[k1], w);
  }
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) { la[17 * k1 + j] = a[k1]; lb[17 * k1 + j] = b[k1]; }
  __syncthreads();
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) { a[n2] = la[17 * j + n2]; b[n2] = lb[17 * j + n2]; }
  dft16<INV>(a);
  dft16<INV>(b);
  __syncthreads();
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) { la[j + 17 * k2] = a[k2]; lb[j + 17 * k2] = b[k2]; }
  __syncthreads();
}

__global__ void __launch_bounds__(v2::NT2, 2) k_fused2(Args A) {
  using namespace v2;
  extern __shared__ __align__(16) unsigned char sm[];
  float2* W = reinterpret_cast<float2*>(sm + OFF_W);
  float2* tw = reinterpret_cast<float2*>(sm + OFF_TW2);
  float2* ex = reinterpret_cast<float2*>(sm + OFF_EX2);
  float* gx = reinterpret_cast<float*>(sm + OFF_GX2);
  float2* ey = reinterpret_cast<float2*>(sm + OFF_EY2);
  float* gy = reinterpret_cast<float*>(sm + OFF_GY2);
  float* kxt = reinterpret_cast<float*>(sm + OFF_KX2);
  float* kyt = reinterpret_cast<float*>(sm + OFF_KY2);
  float* s_ft = reinterpret_cast<float*>(sm + OFF_MISC2);
  float2* s_tf = reinterpret_cast<float2*>(sm + OFF_MISC2 + 7 * RB * 4);
  float2* s_w = reinterpret_cast<float2*>(sm + OFF_MISC2 + 7 * RB * 4 + 56);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + OFF_MISC2 + 7 * RB * 4 + 72);

  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int cid = blockIdx.x / CL;
  const int ncl = gridDim.x / CL;
  const int tid = threadIdx.x;
  const int row0 = rank * RB;
  const size_t plane = (size_t)NX * NY;
  // global slot of the cluster: k_2 .. k_6, y, y low part; k_1 (= k_7 of the previous step)
  // and the local-term stash live in tensor memory, 128 columns each
  float2* slot = A.slots + (size_t)cid * 7 * 2 * plane;
  float2* yg = slot + (size_t)5 * 2 * plane;
  float2* ylo = slot + (size_t)6 * 2 * plane;
  const int warp = tid >> 5;
  if (warp == 0) {
    tmem_alloc(s_tmem, 256);
    tmem_relinquish();
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *s_tmem;
  // this thread's columns: lane quarter warp % 4, column group warp / 4, 8 columns per site pair
  const uint32_t tlane = ((uint32_t)(32 * (warp & 3))) << 16;
  const uint32_t tk1 = tbase + tlane + 64 * (warp >> 2);
  const uint32_t tst = tk1 + 128;

  for (int m = tid; m < 256; m += NT2) {
    double sn, cs;
    sincospi(-2.0 * m / 256.0, &sn, &cs);
    tw[m] = make_float2((float)cs, (float)sn);
  }
  const double dxx = A.Lx / NX, dyy = A.Ly / NY;
  const float inv_n = 1.0f / (float)(NX * NY);
  const double DPc[7] = {0.0, 0.2, 0.3, 0.8, 8.0 / 9.0, 1.0, 1.0};
  const double DPa[7][6] = {{0, 0, 0, 0, 0, 0},
                            {0.2, 0, 0, 0, 0, 0},
                            {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
                            {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
                            {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
                            {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
                            {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};

  for (int si = cid; si < A.n_sec; si += ncl) {
    const Sector S = A.sec[si];
    const FieldDesc& F = A.fd[S.inst];
    for (int i = tid; i < NX; i += NT2) {
      const double xc = -0.5 * A.Lx + i * dxx;
      gx[i] = (float)axis_factor(F, 0, xc);
      double sn, cs;
      sincos(F.pmom[0] * xc, &sn, &cs);
      ex[i] = make_float2((float)cs, (float)sn);
      kxt[i] = (float)(6.283185307179586476925286766559 * (i < NX / 2 ? i : i - NX) / A.Lx);
    }
    for (int i = tid; i < NY; i += NT2)
      kyt[i] = (float)(S.sigma * 6.283185307179586476925286766559 * (i < NY / 2 ? i : i - NY) / A.Ly);
    if (tid < RB) {
      const double yc = -0.5 * A.Ly + (row0 + tid) * dyy;
      gy[tid] = (float)axis_factor(F, 1, yc);
      double sn, cs;
      sincos(F.pmom[1] * yc, &sn, &cs);
      ey[tid] = make_float2((float)cs, (float)sn);
    }
    if (tid < 2) {
      const int c = tid == 0 ? S.c0 : S.c1;
      s_w[tid] = make_float2((float)F.w[2 * c], (float)F.w[2 * c + 1]);
    }
    for (int i = tid; i < NSL; i += NT2) {
      const int comp = i / (RB * NX), rem = i % (RB * NX);
      const size_t gi = comp * plane + (size_t)row0 * NX + rem;
      __stcg(yg + gi, make_float2(0.f, 0.f));
      __stcg(ylo + gi, make_float2(0.f, 0.f));
    }
    __syncthreads();

    const int n_eval = 1 + 6 * A.n_steps;
    for (int ev = 0; ev < n_eval; ++ev) {
      const int step = ev == 0 ? 0 : (ev - 1) / 6;
      const int stage = ev == 0 ? 0 : 1 + (ev - 1) % 6;
      if (ev == 0 || stage == 1) {
        const int st0 = ev == 0 ? 0 : 1, nst = ev == 0 ? 1 : 6;
        if (F.kind == SWF_FIELD_PULSE_GAUSS) {
          if (tid < nst * RB) {
            const int si2 = st0 + tid / RB, r = tid % RB;
            const double ts = A.t_out + step * A.h + DPc[si2] * A.h;
            const double yc = -0.5 * A.Ly + (row0 + r) * dyy;
            s_ft[si2 * RB + r] = (float)time_factor(F, ts, yc);
          } else if (tid >= 128 && tid < 128 + nst) {
            const int si2 = st0 + tid - 128;
            const double ts = A.t_out + step * A.h + DPc[si2] * A.h;
            double sn, cs;
            sincos(F.tsign * F.e0 * ts, &sn, &cs);
            s_tf[si2] = make_float2((float)cs, (float)sn);
          }
        } else if (tid < nst * RB) {
          const int si2 = st0 + tid / RB, r = tid % RB;
          const float4 e = __ldg(A.ttab + ((size_t)S.inst * A.n_steps + step) * 7 + si2);
          s_ft[si2 * RB + r] = e.x;
          if (r == 0) s_tf[si2] = make_float2(e.y, e.z);
        }
        __syncthreads();
      }
      float coef[6];
      const float2* kin[6];
      int nterm = 0;
#pragma unroll
      for (int j = 0; j < 6; ++j) {
        coef[j] = 0.f;
        kin[j] = slot;
      }
      // k_1 comes from tensor memory; k_2 .. k_6 from the global slot
      const float c1 = stage > 0 ? (float)(A.h * DPa[stage][0]) : 0.f;
#pragma unroll
      for (int j = 1; j < 6; ++j) {
        if (j < stage && DPa[stage][j] != 0.0) {
#pragma unroll
          for (int q = 0; q < 6; ++q)
            if (q == nterm) {
              coef[q] = (float)(A.h * DPa[stage][j]);
              kin[q] = slot + (size_t)(j - 1) * 2 * plane;
            }
          ++nterm;
        }
      }
      // stage 0 (k_1) and stage 6 (k_7, the next step's k_1) go to tensor memory
      const bool out_tmem = stage == 0 || stage == 6;
      float2* kout = slot + (size_t)(stage > 0 && stage < 6 ? stage - 1 : 0) * 2 * plane;
      const float2 tf = s_tf[stage];
      const float* ftr = s_ft + stage * RB;
      const float2 w0 = s_w[0], w1 = s_w[1];
      const bool last = stage == 6;
      // ---- 1. stage combine and local term
#pragma unroll 1
      for (int mm = 0; mm < 8; mm += 2) {
        // k_1 of both site pairs of this iteration in one tensor-memory load
        float4 t1a0 = make_float4(0.f, 0.f, 0.f, 0.f), t1a1 = t1a0, t1b0 = t1a0, t1b1 = t1a0;
        if (stage > 0) tmem_ld16(tk1 + 8 * mm, t1a0, t1a1, t1b0, t1b1);
#pragma unroll
      for (int m = mm; m < mm + 2; ++m) {
        const int sp = tid + NT2 * m;
        const int r = sp >> 7;
        const int x = (sp & 127) * 2;
        const size_t g0 = (size_t)(row0 + r) * NX + x;
        const float4 yh0 = __ldcg(reinterpret_cast<const float4*>(yg + g0));
        const float4 yh1 = __ldcg(reinterpret_cast<const float4*>(yg + plane + g0));
        float4 y0 = last ? make_float4(0.f, 0.f, 0.f, 0.f) : yh0;
        float4 y1 = last ? make_float4(0.f, 0.f, 0.f, 0.f) : yh1;
        {
          const float4 k0 = m == mm ? t1a0 : t1b0, k1 = m == mm ? t1a1 : t1b1;
          y0.x = fmaf(c1, k0.x, y0.x); y0.y = fmaf(c1, k0.y, y0.y); y0.z = fmaf(c1, k0.z, y0.z); y0.w = fmaf(c1, k0.w, y0.w);
          y1.x = fmaf(c1, k1.x, y1.x); y1.y = fmaf(c1, k1.y, y1.y); y1.z = fmaf(c1, k1.z, y1.z); y1.w = fmaf(c1, k1.w, y1.w);
        }
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          if (q < nterm) {
            const float4 k0 = __ldcg(reinterpret_cast<const float4*>(kin[q] + g0));
            const float4 k1 = __ldcg(reinterpret_cast<const float4*>(kin[q] + plane + g0));
            const float c = coef[q];
            y0.x = fmaf(c, k0.x, y0.x); y0.y = fmaf(c, k0.y, y0.y); y0.z = fmaf(c, k0.z, y0.z); y0.w = fmaf(c, k0.w, y0.w);
            y1.x = fmaf(c, k1.x, y1.x); y1.y = fmaf(c, k1.y, y1.y); y1.z = fmaf(c, k1.z, y1.z); y1.w = fmaf(c, k1.w, y1.w);
          }
        }
        if (last) {
          float4 l0 = __ldcg(reinterpret_cast<const float4*>(ylo + g0));
          float4 l1 = __ldcg(reinterpret_cast<const float4*>(ylo + plane + g0));
          ff_add(yh0.x, l0.x, y0.x); ff_add(yh0.y, l0.y, y0.y); ff_add(yh0.z, l0.z, y0.z); ff_add(yh0.w, l0.w, y0.w);
          ff_add(yh1.x, l1.x, y1.x); ff_add(yh1.y, l1.y, y1.y); ff_add(yh1.z, l1.z, y1.z); ff_add(yh1.w, l1.w, y1.w);
          __stcg(reinterpret_cast<float4*>(ylo + g0), l0);
          __stcg(reinterpret_cast<float4*>(ylo + plane + g0), l1);
          __stcg(reinterpret_cast<float4*>(yg + g0), y0);
          __stcg(reinterpret_cast<float4*>(yg + plane + g0), y1);
        }
        float2* wa0 = W + r * LD + pidx(x);
        float2* wa1 = W + (RB + r) * LD + pidx(x);
        wa0[0] = make_float2(y0.x, y0.y);
        wa0[1] = make_float2(y0.z, y0.w);
        wa1[0] = make_float2(y1.x, y1.y);
        wa1[1] = make_float2(y1.z, y1.w);
        const float ft = ftr[r];
        const float2 phy = cmul(tf, ey[r]);
        float4 z0, z1;
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const float2 ph = cmul(phy, ex[x + e]);
          const float a = ft * gy[r] * gx[x + e];
          const float2 p0 = (e ? make_float2(y0.z, y0.w) : make_float2(y0.x, y0.y)) + cmul(w0, ph);
          const float2 p1 = (e ? make_float2(y1.z, y1.w) : make_float2(y1.x, y1.y)) + cmul(w1, ph);
          float2 v0, v1;
          sector_v(F.acomp, S.sigma, a, p0, p1, v0, v1);
          v0 = rot<false>(v0);
          v1 = rot<false>(v1);
          if (e) { z0.z = v0.x; z0.w = v0.y; z1.z = v1.x; z1.w = v1.y; }
          else { z0.x = v0.x; z0.y = v0.y; z1.x = v1.x; z1.y = v1.y; }
        }
        tmem_st8(tst + 8 * m, z0, z1);
      }
      }
      tmem_wait_st();
      __syncthreads();
      fft256_lines2<false>(W, tw);
      // ---- 2. rows -> columns (pull into registers, barrier, overwrite in place)
      float2 st[32];
      cluster.sync();
      {
        const int col = tid & 15, r = (tid >> 4) & 15;
#pragma unroll
        for (int comp = 0; comp < 2; ++comp)
#pragma unroll
          for (int i = 0; i < CL; ++i) {
            const int s = (rank + i) & (CL - 1);  // rotated order spreads the reads over the cluster
            st[comp * 16 + i] = cluster.map_shared_rank(W, s)[(comp * RB + r) * LD + pidx(rank * CB + col)];
          }
        cluster.sync();
#pragma unroll
        for (int comp = 0; comp < 2; ++comp)
#pragma unroll
          for (int i = 0; i < CL; ++i) {
            const int s = (rank + i) & (CL - 1);
            W[(comp * CB + col) * LD + pidx(s * RB + r)] = st[comp * 16 + i];
          }
      }
      __syncthreads();
      fft256_lines2<false>(W, tw);
#pragma unroll 4
      for (int m = tid; m < CB * NY; m += NT2) {
        const int col = m >> 8, iy = m & 255;
        const float kx = kxt[rank * CB + col];
        const float ky = kyt[iy];
        float2* pa = W + col * LD + pidx(iy);
        float2* pb = W + (CB + col) * LD + pidx(iy);
        h0_pair(*pa, *pb, kx, ky, inv_n, *pa, *pb);
      }
      __syncthreads();
      fft256_lines2<true>(W, tw);
      // ---- 3. columns -> rows, inverse x-FFT, output
      cluster.sync();
      {
        const int r = tid & 15, col = (tid >> 4) & 15;
#pragma unroll
        for (int comp = 0; comp < 2; ++comp)
#pragma unroll
          for (int i = 0; i < CL; ++i) {
            const int s = (rank + i) & (CL - 1);
            st[comp * 16 + i] = cluster.map_shared_rank(W, s)[(comp * CB + col) * LD + pidx(rank * RB + r)];
          }
        cluster.sync();
#pragma unroll
        for (int comp = 0; comp < 2; ++comp)
#pragma unroll
          for (int i = 0; i < CL; ++i) {
            const int s = (rank + i) & (CL - 1);
            W[(comp * RB + r) * LD + pidx(s * CB + col)] = st[comp * 16 + i];
          }
      }
      __syncthreads();
      fft256_lines2<true>(W, tw);
#pragma unroll 2
      for (int m = 0; m < 8; ++m) {
        const int sp = tid + NT2 * m;
        const int r = sp >> 7;
        const int x = (sp & 127) * 2;
        const size_t g0 = (size_t)(row0 + r) * NX + x;
        float4 z0, z1;
        tmem_ld8(tst + 8 * m, z0, z1);
        const float2* wa0 = W + r * LD + pidx(x);
        const float2* wa1 = W + (RB + r) * LD + pidx(x);
        const float4 o0 = make_float4(wa0[0].x + z0.x, wa0[0].y + z0.y, wa0[1].x + z0.z, wa0[1].y + z0.w);
        const float4 o1 = make_float4(wa1[0].x + z1.x, wa1[0].y + z1.y, wa1[1].x + z1.z, wa1[1].y + z1.w);
        if (out_tmem) {
          tmem_st8(tk1 + 8 * m, o0, o1);
        } else {
          __stcg(reinterpret_cast<float4*>(kout + g0), o0);
          __stcg(reinterpret_cast<float4*>(kout + plane + g0), o1);
        }
      }
      tmem_wait_st();
      __syncthreads();
    }
    float2* out0 = A.psi_out + ((size_t)S.inst * 4 + S.c0) * plane + (size_t)row0 * NX;
    float2* out1 = A.psi_out + ((size_t)S.inst * 4 + S.c1) * plane + (size_t)row0 * NX;
    for (int i = tid; i < RB * NX; i += NT2) {
      out0[i] = __ldcg(yg + (size_t)row0 * NX + i);
      out1[i] = __ldcg(yg + plane + (size_t)row0 * NX + i);
    }
    __syncthreads();
  }
  // no CTA may exit while another CTA of the cluster can still read its shared memory
  cluster.sync();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, 256);
}

// ------------------------------------------------------------------ asynchronous-transpose variant
// The two transposes of an evaluation are pushed by the bulk-copy engine (cp.async.bulk from this
// CTA's shared memory to a peer's, completing on the peer's mbarrier) instead of being pulled by
// the threads, and the threads meanwhile do the work that needs no transposed data: the local
// term of the stage while the forward transpose is in flight, and all but the newest term of the
// next stage combine while the backward one is.  Lines stay in registers where one pass's outputs
// are the next pass's inputs in the same thread: from the inverse x-FFT through k_i and the next
// stage value into the next forward x-FFT, and from the forward y-FFT through H0 (the components
// paired through lane ^ 16) into the inverse y-FFT.  The arithmetic is that of `k_fused`, in the
// same order; only the data movement differs.
//
// Both exchange buffers are 2 x 16 chunks of 16 x 16 values: chunk (c, a) of component c holds, in
// the row buffer X1, the 16 rows of this CTA at x in [16 a, 16 a + 16), and in the column buffer
// X2, the 16 columns of this CTA at y in [16 a, 16 a + 16).  Chunk (c, s) of one CTA is exactly
// chunk (c, rank) of CTA s after the transpose, so each transpose is 32 contiguous 2 KB copies per
// CTA.  Inside a chunk, row b keeps its 16 values at positions d ^ b (an XOR swizzle written by the
// producer and kept by the copy), so that every FFT pass reads and writes without bank conflicts.
//
// Ordering.  Each CTA arms its receive barrier for a transpose before it arrives at the cluster
// barrier that lets the senders start, and arrives only after its previous receive completed; a
// sender waits at that cluster barrier before it copies.  So every copy finds its destination free
// (all copies of the previous use, and the receiver's reads, are complete) and its barrier armed.
// Every wait is bounded: a CTA whose copies do not arrive in about half a second sets the
// launch's status word, stops copying and waiting, keeps to the cluster barriers (so that no peer
// is left waiting there), and writes NaN for its rows of the sector, so that the failure shows in
// the result as well.
namespace v3 {
constexpr int CHK = 256;                    // complex values in one chunk
constexpr int NBUF = 2 * CL * CHK;          // complex values in one exchange buffer
constexpr uint32_t XBYTES = NBUF * 8;       // bytes received per transpose
constexpr int OFF_X1 = 0;                   // rows, chunk (c, x / 16), row, x % 16
constexpr int OFF_X2 = OFF_X1 + NBUF * 8;   // columns, chunk (c, y / 16), y % 16, column
constexpr int OFF_Y3 = OFF_X2 + NBUF * 8;   // state y, two sites per float4 at [k2 / 2][thread]
constexpr int OFF_TW3 = OFF_Y3 + NSL * 8;
constexpr int OFF_EX3 = OFF_TW3 + 256 * 8;
constexpr int OFF_GX3 = OFF_EX3 + NX * 8;
constexpr int OFF_EY3 = OFF_GX3 + NX * 4;
constexpr int OFF_GY3 = OFF_EY3 + RB * 8;
constexpr int OFF_KX3 = OFF_GY3 + RB * 4;
constexpr int OFF_KY3 = OFF_KX3 + NX * 4;
constexpr int OFF_MISC3 = OFF_KY3 + NY * 4;
constexpr int OFF_BAR3 = OFF_MISC3 + 7 * RB * 4 + 7 * 8 + 16 + 16;  // two mbarriers
constexpr int SMEM3 = OFF_BAR3 + 16;
constexpr long long WAIT3 = 1ll << 30;  // cycles before a receive wait gives up
static_assert(OFF_BAR3 % 8 == 0, "mbarrier alignment");
static_assert(OFF_X2 % 16 == 0 && OFF_X1 % 16 == 0, "bulk-copy alignment");
static_assert(SMEM3 <= 227 * 1024, "shared memory");
}  // namespace v3

// position of value (c, a, b, d) in an exchange buffer: chunk (c, a), row b, column d ^ b
__host__ __device__ __forceinline__ int q3(int c, int a, int b, int d) {
  return ((((c << 4) + a) << 4) + b) * 16 + (d ^ b);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
// the address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t peer_addr(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void bulk_push(uint32_t dst, uint32_t src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   dst),
               "r"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void mbar_init3(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arm3(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// waits for the phase of the given parity to complete; false after WAIT3 cycles
__device__ __forceinline__ bool mbar_wait3(uint32_t bar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > v3::WAIT3) return false;
  }
}
__device__ __forceinline__ void cl_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cl_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }
// generic-proxy writes of this thread become visible to the bulk-copy engine
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 256-point FFTs of the 32 rows (both components) of X1 along x, in place, are the same two
// radix-16 passes as fft256_lines.  Pass 1: thread (c, row, j) transforms x = 16 n1 + j; pass 2:
// thread (c, jj, row) transforms x = 16 jj + n2 and writes x = jj + 16 k2.  twp[16 k1 + j] holds
// the twiddle W256^(j k1) of pass 1 (consecutive for the 16 values of j that a half-warp reads).
//
// Row lines kept in registers between the inverse x-FFT of one evaluation and the forward x-FFT
// of the next.  Thread t owns the 16 sites (c, row, x = jj + 16 k2), k2 = 0..15, of
// c = (t >> 4) & 1, row = t & 15, jj = t >> 5: the outputs of its last inverse pass and the
// inputs of its next forward first pass.  Its tensor-memory columns 2 k2, 2 k2 + 1 hold site k2
// of each slab; the state y (shared memory) and the cluster's global slots keep two sites per
// float4 at [k2 / 2][t], so every access of a warp is contiguous.  The partner component of a
// site is lane ^ 16 of the same warp.
__device__ __forceinline__ int own_c() { return (threadIdx.x >> 4) & 1; }
__device__ __forceinline__ int own_row() { return threadIdx.x & 15; }
__device__ __forceinline__ int own_jj() { return threadIdx.x >> 5; }

// forward x-FFT of the rows, pass 1 from the registers a[k2] (x = jj + 16 k2 = 16 n1 + j with
// j = jj), pass 2 with thread (c, jj, row) = (t >> 8, (t >> 4) & 15, t & 15); the caller
// synchronises after
__device__ __forceinline__ void fft_rows3_from_regs(float2* X, const float2* twp, float2 (&a)[16]) {
  const int t = threadIdx.x;
  {
    const int c = own_c(), row = own_row(), j = own_jj();
    dft16<false>(a);
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) a[k1] = cmul(a[k1], twp[k1 * 16 + j]);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) X[q3(c, k1, row, j)] = a[k1];
  }
  __syncthreads();
  const int c = t >> 8, jj = (t >> 4) & 15, row = t & 15;
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) a[n2] = X[q3(c, jj, row, n2)];
  dft16<false>(a);
  __syncthreads();
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) X[q3(c, k2, row, jj)] = a[k2];
}

// inverse x-FFT of the rows, pass 1 with thread (c, row, j) = (t >> 8, (t >> 4) & 15, t & 15),
// pass 2 into the registers a[k2] of the owning thread; ends with a barrier (every thread has
// read X before anyone writes it again)
__device__ __forceinline__ void fft_rows3_to_regs(float2* X, const float2* twp, float2 (&a)[16]) {
  const int t = threadIdx.x;
  {
    const int c = t >> 8, row = (t >> 4) & 15, j = t & 15;
#pragma unroll
    for (int n1 = 0; n1 < 16; ++n1) a[n1] = X[q3(c, n1, row, j)];
    dft16<true>(a);
#pragma unroll
    for (int k1 = 1; k1 < 16; ++k1) a[k1] = cmulc(a[k1], twp[k1 * 16 + j]);
#pragma unroll
    for (int k1 = 0; k1 < 16; ++k1) X[q3(c, k1, row, j)] = a[k1];
  }
  __syncthreads();
  const int c = own_c(), row = own_row(), jj = own_jj();
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) a[n2] = X[q3(c, jj, row, n2)];
  dft16<true>(a);
  __syncthreads();
}

// The column side of an evaluation in one pass over X2: forward 256-point y-FFT of the 32 columns
// (two radix-16 passes as fft256_lines, y = 16 n1 + j then y = 16 j + n2), -i H0(kappa)/N per
// mode (kxc: kappa_x of this CTA's columns, kyt: sigma kappa_y per mode), inverse y-FFT.
// Thread t = (j = t >> 5, c = (t >> 4) & 1, col = t & 15): the outputs y = j + 16 k2 of its forward
// pass 2 are the inputs y = 16 n1 + j of its inverse pass 1, and the other component of each mode
// is lane ^ 16, so H0 is applied in registers.  The caller synchronises after.
__device__ __forceinline__ void fft_cols3_h0(float2* X, const float2* twp, const float* kxc, const float* kyt,
                                             float inv_n) {
  const int t = threadIdx.x, col = t & 15, c = (t >> 4) & 1, j = t >> 5;
  float2 a[16];
#pragma unroll
  for (int n1 = 0; n1 < 16; ++n1) a[n1] = X[q3(c, n1, j, col)];
  dft16<false>(a);
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) a[k1] = cmul(a[k1], twp[k1 * 16 + j]);
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) X[q3(c, k1, j, col)] = a[k1];
  __syncthreads();
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) a[n2] = X[q3(c, j, n2, col)];
  dft16<false>(a);
  const float kx = kxc[col];
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) {
    const float2 own = a[k2];
    const float2 oth = make_float2(__shfl_xor_sync(0xffffffffu, own.x, 16), __shfl_xor_sync(0xffffffffu, own.y, 16));
    float2 o0, o1;
    h0_pair(c ? oth : own, c ? own : oth, kx, kyt[j + 16 * k2], inv_n, o0, o1);
    a[k2] = c ? o1 : o0;
  }
  dft16<true>(a);
#pragma unroll
  for (int k1 = 1; k1 < 16; ++k1) a[k1] = cmulc(a[k1], twp[k1 * 16 + j]);
  __syncthreads();  // every thread has read its forward pass-2 inputs
#pragma unroll
  for (int k1 = 0; k1 < 16; ++k1) X[q3(c, k1, j, col)] = a[k1];
  __syncthreads();
#pragma unroll
  for (int n2 = 0; n2 < 16; ++n2) a[n2] = X[q3(c, j, n2, col)];
  dft16<true>(a);
  __syncthreads();
#pragma unroll
  for (int k2 = 0; k2 < 16; ++k2) X[q3(c, k2, j, col)] = a[k2];
}

__device__ __forceinline__ float4 shfl16(float4 v) {
  return make_float4(__shfl_xor_sync(0xffffffffu, v.x, 16), __shfl_xor_sync(0xffffffffu, v.y, 16),
                     __shfl_xor_sync(0xffffffffu, v.z, 16), __shfl_xor_sync(0xffffffffu, v.w, 16));
}

__global__ void __launch_bounds__(NT, 1) k_fused3(Args A) {
  using namespace v3;
  extern __shared__ __align__(16) unsigned char sm[];
  float2* X1 = reinterpret_cast<float2*>(sm + OFF_X1);
  float2* X2 = reinterpret_cast<float2*>(sm + OFF_X2);
  float4* Ys4 = reinterpret_cast<float4*>(sm + OFF_Y3);  // [k2 / 2][t]: the sites this thread owns
  float2* twp = reinterpret_cast<float2*>(sm + OFF_TW3);  // [k1][j]: W256^(j k1)
  float2* ex = reinterpret_cast<float2*>(sm + OFF_EX3);
  float* gx = reinterpret_cast<float*>(sm + OFF_GX3);
  float2* ey = reinterpret_cast<float2*>(sm + OFF_EY3);
  float* gy = reinterpret_cast<float*>(sm + OFF_GY3);
  float* kxt = reinterpret_cast<float*>(sm + OFF_KX3);
  float* kyt = reinterpret_cast<float*>(sm + OFF_KY3);
  float* s_ft = reinterpret_cast<float*>(sm + OFF_MISC3);
  float2* s_tf = reinterpret_cast<float2*>(sm + OFF_MISC3 + 7 * RB * 4);
  float2* s_w = reinterpret_cast<float2*>(sm + OFF_MISC3 + 7 * RB * 4 + 56);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + OFF_MISC3 + 7 * RB * 4 + 72);
  const uint32_t bar_f = smem_u32(sm + OFF_BAR3), bar_b = bar_f + 8;
  const uint32_t x1a = smem_u32(X1), x2a = smem_u32(X2);

  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int cid = blockIdx.x / CL;
  const int ncl = gridDim.x / CL;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int row0 = rank * RB;
  const size_t plane = (size_t)NX * NY;
  // the cluster's global slots k_4, k_5, k_6 and the low part of y; this CTA's part of each,
  // two of this thread's sites per float4 at [k2 / 2][t]
  float4* slot4 = reinterpret_cast<float4*>(A.slots + (size_t)cid * 4 * 2 * plane) + (size_t)rank * (NSL / 2);
  const size_t sstride = plane;  // float4 per slot (2 plane complex values)
  float4* ylo4 = slot4 + 3 * sstride;
  if (warp == 0) {
    tmem_alloc(s_tmem, 512);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init3(bar_f, 1);
    mbar_init3(bar_b, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int m = tid; m < 256; m += NT) {
    const int k1 = m >> 4, j = m & 15;
    double s, c;
    sincospi(-2.0 * ((j * k1) & 255) / 256.0, &s, &c);
    twp[m] = make_float2((float)c, (float)s);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tbase = *s_tmem;
  const uint32_t tme = tbase + (((uint32_t)(32 * (warp & 3))) << 16) + 32 * (warp >> 2);
  const uint32_t tstash = tme + 128 * 3;
  if (tid == 0) mbar_arm3(bar_f, XBYTES);  // the first forward transpose
  cl_arrive();                             // barriers initialised and armed
  uint32_t par_f = 0, par_b = 0;
  bool err = false;
  // lane L of warp 0 copies chunk (L / 16, peer) to peer (rank + L) % 16
  const int cc = lane >> 4, peer = (rank + (lane & 15)) & (CL - 1);
  // the sites this thread owns
  const int oc = own_c(), orow = own_row(), ojj = own_jj();

  const double dxx = A.Lx / NX, dyy = A.Ly / NY;
  const float inv_n = 1.0f / (float)(NX * NY);
  const double DPc[7] = {0.0, 0.2, 0.3, 0.8, 8.0 / 9.0, 1.0, 1.0};
  const double DPa[7][6] = {{0, 0, 0, 0, 0, 0},
                            {0.2, 0, 0, 0, 0, 0},
                            {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
                            {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
                            {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
                            {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
                            {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};

  for (int si = cid; si < A.n_sec; si += ncl) {
    const Sector S = A.sec[si];
    const FieldDesc& F = A.fd[S.inst];
    for (int i = tid; i < NX; i += NT) {
      const double xc = -0.5 * A.Lx + i * dxx;
      gx[i] = (float)axis_factor(F, 0, xc);
      double s, c;
      sincos(F.pmom[0] * xc, &s, &c);
      ex[i] = make_float2((float)c, (float)s);
    }
    if (tid < RB) {
      const double yc = -0.5 * A.Ly + (row0 + tid) * dyy;
      gy[tid] = (float)axis_factor(F, 1, yc);
      double s, c;
      sincos(F.pmom[1] * yc, &s, &c);
      ey[tid] = make_float2((float)c, (float)s);
    }
    for (int i = tid; i < NX; i += NT) kxt[i] = (float)(6.283185307179586476925286766559 * (i < NX / 2 ? i : i - NX) / A.Lx);
    for (int i = tid; i < NY; i += NT)
      kyt[i] = (float)(S.sigma * 6.283185307179586476925286766559 * (i < NY / 2 ? i : i - NY) / A.Ly);
    if (tid < 2) {
      const int c = tid == 0 ? S.c0 : S.c1;
      s_w[tid] = make_float2((float)F.w[2 * c], (float)F.w[2 * c + 1]);
    }
    // y = 0, its low part 0, and the first stage value Y = y = 0 in registers and in the stash
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int h = 0; h < 8; ++h) {
      Ys4[h * NT + tid] = z4;
      __stcg(ylo4 + h * NT + tid, z4);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) tmem_st8(tstash + 8 * q, z4, z4);
    tmem_wait_st();
    float2 a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[k] = make_float2(0.f, 0.f);
    __syncthreads();

    const int n_eval = 1 + 6 * A.n_steps;
    for (int ev = 0; ev < n_eval; ++ev) {
      const int step = ev == 0 ? 0 : (ev - 1) / 6;
      const int stage = ev == 0 ? 0 : 1 + (ev - 1) % 6;
      if (ev == 0 || stage == 1) {
        const int st0 = ev == 0 ? 0 : 1, nst = ev == 0 ? 1 : 6;
        if (F.kind == SWF_FIELD_PULSE_GAUSS) {
          if (tid < nst * RB) {
            const int si2 = st0 + tid / RB, r = tid % RB;
            const double ts = A.t_out + step * A.h + DPc[si2] * A.h;
            const double yc = -0.5 * A.Ly + (row0 + r) * dyy;
            s_ft[si2 * RB + r] = (float)time_factor(F, ts, yc);
          } else if (tid >= 128 && tid < 128 + nst) {
            const int si2 = st0 + tid - 128;
            const double ts = A.t_out + step * A.h + DPc[si2] * A.h;
            double s, c;
            sincos(F.tsign * F.e0 * ts, &s, &c);
            s_tf[si2] = make_float2((float)c, (float)s);
          }
        } else if (tid < nst * RB) {
          const int si2 = st0 + tid / RB, r = tid % RB;
          const float4 e = __ldg(A.ttab + ((size_t)S.inst * A.n_steps + step) * 7 + si2);
          s_ft[si2 * RB + r] = e.x;
          if (r == 0) s_tf[si2] = make_float2(e.y, e.z);
        }
        __syncthreads();
      }

      // ---- forward x-FFT of the stage value Y (registers), then push chunk (c, s) to CTA s
      fft_rows3_from_regs(X1, twp, a);
      fence_async_smem();
      __syncthreads();
      cl_wait();  // every CTA's X2 is free and its receive barrier armed
      if (warp == 0 && !__any_sync(0xffffffffu, err) && !A.drop)
        bulk_push(peer_addr(x2a + (uint32_t)((cc * CL + rank) * CHK * 8), peer),
                  x1a + (uint32_t)((cc * CL + peer) * CHK * 8), CHK * 8, peer_addr(bar_f, peer));

      // ---- meanwhile: local term Z = -i V (Y + psi_b) of this stage, from the stash (Y, both
      // components through the partner lane) to the stash
      {
        const float2 tf = s_tf[stage];
        const float ft = s_ft[stage * RB + orow];
        const float2 w0 = s_w[0], w1 = s_w[1];
        const float2 phy = cmul(tf, ey[orow]);
        const float fg = ft * gy[orow];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float4 ya, yb;
          tmem_ld8(tstash + 8 * q, ya, yb);
          const float4 pa = shfl16(ya), pb = shfl16(yb);
          float2 z[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int x = ojj + 16 * (4 * q + e);
            const float4& yo = e < 2 ? ya : yb;
            const float4& yp = e < 2 ? pa : pb;
            const float2 own = (e & 1) ? make_float2(yo.z, yo.w) : make_float2(yo.x, yo.y);
            const float2 oth = (e & 1) ? make_float2(yp.z, yp.w) : make_float2(yp.x, yp.y);
            const float2 y0 = oc ? oth : own, y1 = oc ? own : oth;
            const float2 ph = cmul(phy, ex[x]);
            const float av = fg * gx[x];
            const float2 p0 = y0 + cmul(w0, ph);
            const float2 p1 = y1 + cmul(w1, ph);
            float2 v0, v1;
            sector_v(F.acomp, S.sigma, av, p0, p1, v0, v1);
            z[e] = rot<false>(oc ? v1 : v0);
          }
          tmem_st8(tstash + 8 * q, make_float4(z[0].x, z[0].y, z[1].x, z[1].y), make_float4(z[2].x, z[2].y, z[3].x, z[3].y));
        }
        tmem_wait_st();
      }
      {
        // every thread waits for the forward copies itself (no block barrier after the wait)
        const bool bad = !err && !mbar_wait3(bar_f, par_f);
        if (tid == 0 && !err) {
          if (!bad) mbar_arm3(bar_b, XBYTES);  // for the backward transpose of this evaluation
          else if (A.status) atomicOr(A.status, 1);
        }
        err = err || bad;
        par_f ^= 1u;
      }
      cl_arrive();  // the forward copies into this CTA are complete

      // ---- columns: forward y-FFT, -i H0(kappa)/N per mode in registers, inverse y-FFT; push
      // chunk (c, s) back
      fft_cols3_h0(X2, twp, kxt + rank * CB, kyt, inv_n);
      fence_async_smem();
      __syncthreads();
      cl_wait();  // every CTA's X1 is free and its receive barrier armed
      if (warp == 0 && !__any_sync(0xffffffffu, err) && !A.drop)
        bulk_push(peer_addr(x1a + (uint32_t)((cc * CL + rank) * CHK * 8), peer),
                  x2a + (uint32_t)((cc * CL + peer) * CHK * 8), CHK * 8, peer_addr(bar_b, peer));

      // ---- meanwhile: the next stage combine without its newest term, P = y + h sum_{j < new} a_j k_j
      // (h sum b_j k_j without y before the last stage), in the order of k_fused
      const bool has_next = ev + 1 < n_eval;
      const int nxt = stage == 6 ? 1 : stage + 1;  // the next stage (stage 0 is followed by 1)
      const int jn = nxt - 1;                      // index of the newest k (the one computed now)
      const bool nlast = nxt == 6;
      float4 P[8];
      if (has_next) {
        const int ntp = jn < 3 ? jn : 3;  // tensor-memory terms before the newest
        float ct[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) ct[j] = (j < ntp) ? (float)(A.h * DPa[nxt][j]) : 0.f;
        float coef[2];
        const float4* kin[2];
        int nterm = 0;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          coef[j] = 0.f;
          kin[j] = slot4;
        }
#pragma unroll
        for (int j = 3; j < 5; ++j) {
          if (j < jn && DPa[nxt][j] != 0.0) {
#pragma unroll
            for (int q = 0; q < 2; ++q)
              if (q == nterm) {
                coef[q] = (float)(A.h * DPa[nxt][j]);
                kin[q] = slot4 + (size_t)(j - 3) * sstride;
              }
            ++nterm;
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float4 y0 = make_float4(0.f, 0.f, 0.f, 0.f), y1 = y0;
          if (!nlast) {
            y0 = Ys4[(2 * q) * NT + tid];
            y1 = Ys4[(2 * q + 1) * NT + tid];
          }
          if (ntp > 0) {
            uint32_t tr[3][8];
#pragma unroll
            for (int j = 0; j < 3; ++j)
              if (j < ntp) tmem_ld8_nowait(tme + 128 * j + 8 * q, tr[j]);
            tmem_wait_ld();
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              if (j < ntp) {
                const float2 c = make_float2(ct[j], ct[j]);
                fma4(c, make_float4(__uint_as_float(tr[j][0]), __uint_as_float(tr[j][1]), __uint_as_float(tr[j][2]),
                                    __uint_as_float(tr[j][3])), y0);
                fma4(c, make_float4(__uint_as_float(tr[j][4]), __uint_as_float(tr[j][5]), __uint_as_float(tr[j][6]),
                                    __uint_as_float(tr[j][7])), y1);
              }
            }
          }
#pragma unroll
          for (int qq = 0; qq < 2; ++qq) {
            if (qq < nterm) {
              const float4 k0 = __ldcg(kin[qq] + (2 * q) * NT + tid);
              const float4 k1 = __ldcg(kin[qq] + (2 * q + 1) * NT + tid);
              const float2 c = make_float2(coef[qq], coef[qq]);
              fma4(c, k0, y0);
              fma4(c, k1, y1);
            }
          }
          P[2 * q] = y0;
          P[2 * q + 1] = y1;
        }
      }
      {
        const bool bad = !err && !mbar_wait3(bar_b, par_b);
        if (tid == 0 && !err) {
          if (!bad) mbar_arm3(bar_f, XBYTES);  // for the next forward transpose
          else if (A.status) atomicOr(A.status, 1);
        }
        err = err || bad;
        par_b ^= 1u;
      }
      cl_arrive();  // the backward copies into this CTA are complete

      // ---- inverse x-FFT into registers; k = (that) + Z; the next stage value Y' = P + h a_new k
      fft_rows3_to_regs(X1, twp, a);
      {
        const int oslab = stage == 0 || stage == 6 ? 0 : (stage <= 2 ? stage : -1);
        float4* kout = slot4 + (size_t)(stage >= 3 && stage <= 5 ? stage - 3 : 0) * sstride;
        const bool use_new = jn < 3 || DPa[nxt][jn] != 0.0;
        const float cnv = (float)(A.h * DPa[nxt][jn]);
        const float2 cn = make_float2(cnv, cnv);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float4 za, zb;
          tmem_ld8(tstash + 8 * q, za, zb);
          const float4 o0 = make_float4(a[4 * q].x + za.x, a[4 * q].y + za.y, a[4 * q + 1].x + za.z, a[4 * q + 1].y + za.w);
          const float4 o1 = make_float4(a[4 * q + 2].x + zb.x, a[4 * q + 2].y + zb.y, a[4 * q + 3].x + zb.z, a[4 * q + 3].y + zb.w);
          if (oslab >= 0) {
            tmem_st8(tme + 128 * oslab + 8 * q, o0, o1);
          } else {
            __stcg(kout + (2 * q) * NT + tid, o0);
            __stcg(kout + (2 * q + 1) * NT + tid, o1);
          }
          if (has_next) {
            float4 y0 = P[2 * q], y1 = P[2 * q + 1];
            if (use_new) {
              fma4(cn, o0, y0);
              fma4(cn, o1, y1);
            }
            if (nlast) {
              // y_new = y + h sum_j b_j k_j in float-float
              const float4 yh0 = Ys4[(2 * q) * NT + tid];
              const float4 yh1 = Ys4[(2 * q + 1) * NT + tid];
              float4 l0 = __ldcg(ylo4 + (2 * q) * NT + tid);
              float4 l1 = __ldcg(ylo4 + (2 * q + 1) * NT + tid);
              ff_add(yh0.x, l0.x, y0.x); ff_add(yh0.y, l0.y, y0.y); ff_add(yh0.z, l0.z, y0.z); ff_add(yh0.w, l0.w, y0.w);
              ff_add(yh1.x, l1.x, y1.x); ff_add(yh1.y, l1.y, y1.y); ff_add(yh1.z, l1.z, y1.z); ff_add(yh1.w, l1.w, y1.w);
              __stcg(ylo4 + (2 * q) * NT + tid, l0);
              __stcg(ylo4 + (2 * q + 1) * NT + tid, l1);
              Ys4[(2 * q) * NT + tid] = y0;
              Ys4[(2 * q + 1) * NT + tid] = y1;
            }
            tmem_st8(tstash + 8 * q, y0, y1);
            a[4 * q] = make_float2(y0.x, y0.y);
            a[4 * q + 1] = make_float2(y0.z, y0.w);
            a[4 * q + 2] = make_float2(y1.x, y1.y);
            a[4 * q + 3] = make_float2(y1.z, y1.w);
          }
        }
        tmem_wait_st();
      }
    }
    // psi(t_in) of the sector into the 4-component output (NaN if a transpose failed)
    err = __syncthreads_or(err);
    {
      const float2 nan2 = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
      float2* out = A.psi_out + ((size_t)S.inst * 4 + (oc ? S.c1 : S.c0)) * plane + (size_t)(row0 + orow) * NX + ojj;
#pragma unroll
      for (int h = 0; h < 8; ++h) {
        const float4 v = Ys4[h * NT + tid];
        out[16 * (2 * h)] = err ? nan2 : make_float2(v.x, v.y);
        out[16 * (2 * h + 1)] = err ? nan2 : make_float2(v.z, v.w);
      }
    }
    __syncthreads();
  }
  if (err) {  // let copies that were still under way land before the cluster lets this CTA go
    const long long t0 = clock64();
    while (clock64() - t0 < 20000000ll) {
    }
  }
  cl_wait();  // every copy of the last transposes is complete
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, 512);
}

}  // namespace fused

// True when the fused kernel covers this march: (2+1)D 256 x 256 grid, complex64, no
// momentum along the trivial z axis, and fields that keep the z-spin sectors apart.
bool fused_applicable(const GridDesc& g, int n_f, const FieldDesc* fd, swf_precision prec) {
  if (prec != SWF_C64) return false;
  if (g.n[0] != fused::NX || g.n[1] != fused::NY || g.n[2] != 1) return false;
  for (int f = 0; f < n_f; ++f) {
    if (fd[f].K[2] != 0.0) return false;
    if (fd[f].acomp == 3) return false;
  }
  return true;
}

static int g_fused_clusters[64][3];  // per device and variant: resident clusters + 1 (0: not set up)

// Kernel attributes and the number of clusters that can be resident at once (cached per device).
static swf_status fused_setup(int var, cudaStream_t st) {
  using namespace fused;
  void (*kern)(Args) = var == 2 ? k_fused3 : var == 1 ? k_fused2 : k_fused;
  const int nthr = var == 1 ? v2::NT2 : NT;
  const int smem = var == 2 ? v3::SMEM3 : var == 1 ? v2::SMEM2 : SMEM;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return cuda_status(e, "cluster size attribute");
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return cuda_status(e, "shared memory attribute");
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(CL, 1, 1);
  cfg.blockDim = dim3(nthr, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at;
  at.id = cudaLaunchAttributeClusterDimension;
  at.val.clusterDim.x = CL;
  at.val.clusterDim.y = 1;
  at.val.clusterDim.z = 1;
  cfg.attrs = &at;
  cfg.numAttrs = 1;
  int ncl = 0;
  e = cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg);
  if (e != cudaSuccess) return cuda_status(e, "cudaOccupancyMaxActiveClusters");
  g_fused_clusters[dev_slot()][var] = (ncl > 0 ? ncl : 0) + 1;
  return SWF_OK;
}

int fused_resident_clusters(swf_ctx* ctx) {
  const int var = ctx->fused_variant - 1;
  if (g_fused_clusters[dev_slot()][var] == 0 && fused_setup(var, ctx->stream) != SWF_OK) return 0;
  return g_fused_clusters[dev_slot()][var] - 1;
}

swf_status march_fused(swf_ctx* ctx, const GridDesc& g, double t_in, double t_out, int n_steps, int n_f,
                       const FieldDesc* fd_host, void* psi_out, cudaStream_t st) {
  using namespace fused;
  const int var = ctx->fused_variant - 1;
  void (*kern)(Args) = var == 2 ? k_fused3 : var == 1 ? k_fused2 : k_fused;
  const int nthr = var == 1 ? v2::NT2 : NT;
  const int smem = var == 2 ? v3::SMEM3 : var == 1 ? v2::SMEM2 : SMEM;
  const int narr = var == 1 ? 7 : 4;
  cudaError_t e;
  auto config = [&](int ncl, cudaLaunchAttribute* at) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ncl * CL, 1, 1);
    cfg.blockDim = dim3(nthr, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    at->id = cudaLaunchAttributeClusterDimension;
    at->val.clusterDim.x = CL;
    at->val.clusterDim.y = 1;
    at->val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
  };
  int* ncl_slot = &g_fused_clusters[dev_slot()][var];
  if (*ncl_slot == 0) {
    swf_status s0 = fused_setup(var, st);
    if (s0 != SWF_OK) return s0;
  }
  if (*ncl_slot < 2) {
    set_error("the fused march kernel cannot be resident on this device");
    return SWF_EUNSUPPORTED;
  }
  const int n_sec = 2 * n_f;
  const int ncl = *ncl_slot - 1 < n_sec ? *ncl_slot - 1 : n_sec;
  const size_t plane = (size_t)NX * NY;
  swf_status s;
  void *pfd, *psec, *pslots;
  if ((s = ws_get(ctx, "fused.fd", sizeof(FieldDesc) * n_f, &pfd)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "fused.sec", sizeof(Sector) * n_sec, &psec)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "fused.slots", (size_t)ncl * narr * 2 * plane * sizeof(float2), &pslots)) != SWF_OK) return s;
  std::vector<Sector> sec(n_sec);
  for (int f = 0; f < n_f; ++f) {
    sec[2 * f] = {f, 0, 3, +1};
    sec[2 * f + 1] = {f, 1, 2, -1};
  }
  e = cudaMemcpyAsync(pfd, fd_host, sizeof(FieldDesc) * n_f, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "upload field descriptors");
  e = cudaMemcpyAsync(psec, sec.data(), sizeof(Sector) * n_sec, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "upload sector table");
  e = cudaStreamSynchronize(st);  // the sector table is a host temporary; the march itself runs on
  if (e != cudaSuccess) return cuda_status(e, "upload sector table");  // after this call returns
  void* ptab;
  if ((s = ws_get(ctx, "fused.ttab", (size_t)n_f * n_steps * 7 * sizeof(float4), &ptab)) != SWF_OK) return s;
  {
    ProfScope ps(ctx, "k_time_table", st);
    const size_t total = (size_t)n_f * n_steps * 7;
    const int nb = (int)((total + 255) / 256 < 4096 ? (total + 255) / 256 : 4096);
    k_time_table<<<nb, 256, 0, st>>>((const FieldDesc*)pfd, n_f, n_steps, t_out, (t_in - t_out) / n_steps,
                                     (float4*)ptab);
  }
  void* pstatus;
  if ((s = ws_get(ctx, "fused.status", sizeof(int), &pstatus)) != SWF_OK) return s;
  e = cudaMemsetAsync(pstatus, 0, sizeof(int), st);
  if (e != cudaSuccess) return cuda_status(e, "clear the fused kernel's status");
  ctx->fused_status_dev = (int*)pstatus;
  Args A;
  A.status = (int*)pstatus;
  A.drop = var == 2 ? ctx->fused_drop : 0;
  A.ttab = (const float4*)ptab;
  A.fd = (const FieldDesc*)pfd;
  A.sec = (const Sector*)psec;
  A.n_sec = n_sec;
  A.slots = (float2*)pslots;
  A.psi_out = (float2*)psi_out;
  A.Lx = g.L[0];
  A.Ly = g.L[1];
  A.t_out = t_out;
  A.h = (t_in - t_out) / n_steps;
  A.n_steps = n_steps;
  cudaLaunchAttribute at;
  cudaLaunchConfig_t cfg = config(ncl, &at);
  {
    ProfScope ps(ctx, var == 2 ? "k_fused3" : var == 1 ? "k_fused2" : "k_fused", st);
    e = cudaLaunchKernelEx(&cfg, kern, A);
  }
  if (e != cudaSuccess) return cuda_status(e, "launch fused march");
  ctx->fields_fused += n_f;
  return SWF_OK;
}


}  // namespace swf
