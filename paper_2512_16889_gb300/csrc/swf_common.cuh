// Shared device helpers of the SWF march: complex arithmetic, small DFT butterflies and a
// shared-memory Stockham pass for the pseudo-spectral derivative (Sec. II.A, Eq. 10).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace swf {

template <typename R>
struct alignas(2 * sizeof(R)) cpx {
  R x, y;
};

template <typename R> __host__ __device__ __forceinline__ cpx<R> mk(R a, R b) { cpx<R> c; c.x = a; c.y = b; return c; }
template <typename R> __host__ __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
template <typename R> __host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
template <typename R> __host__ __device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename R> __host__ __device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) { return mk<R>(s * a.x, s * a.y); }
template <typename R> __host__ __device__ __forceinline__ cpx<R> cconj(cpx<R> a) { return mk<R>(a.x, -a.y); }
// multiply by +i and by -i
template <typename R> __host__ __device__ __forceinline__ cpx<R> mul_i(cpx<R> a) { return mk<R>(-a.y, a.x); }
template <typename R> __host__ __device__ __forceinline__ cpx<R> mul_mi(cpx<R> a) { return mk<R>(a.y, -a.x); }
// conj(a) * b
template <typename R> __host__ __device__ __forceinline__ cpx<R> cdot(cpx<R> a, cpx<R> b) {
  return mk<R>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// Complex arithmetic with every rounding fixed: built from the _rn intrinsics, which the compiler
// neither fuses into multiply-adds nor reorders.  Code that several kernels inline and whose
// results must agree bit for bit between them (the Breit-Wheeler integrand of single-photon,
// photon-scan and multi-grid launches) uses these instead of the operators above.
__device__ __forceinline__ float rn_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rn_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rn_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rn_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rn_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rn_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename R> __device__ __forceinline__ cpx<R> xadd(cpx<R> a, cpx<R> b) {
  return mk<R>(rn_add(a.x, b.x), rn_add(a.y, b.y));
}
template <typename R> __device__ __forceinline__ cpx<R> xmul(cpx<R> a, cpx<R> b) {
  return mk<R>(rn_fma(a.x, b.x, -rn_mul(a.y, b.y)), rn_fma(a.x, b.y, rn_mul(a.y, b.x)));
}
template <typename R> __device__ __forceinline__ cpx<R> xscale(R s, cpx<R> a) {
  return mk<R>(rn_mul(s, a.x), rn_mul(s, a.y));
}
// conj(a) b
template <typename R> __device__ __forceinline__ cpx<R> xcdot(cpx<R> a, cpx<R> b) {
  return mk<R>(rn_fma(a.x, b.x, rn_mul(a.y, b.y)), rn_fma(a.x, b.y, -rn_mul(a.y, b.x)));
}
template <typename Rto, typename Rfrom> __host__ __device__ __forceinline__ cpx<Rto> cvt(cpx<Rfrom> a) {
  return mk<Rto>((Rto)a.x, (Rto)a.y);
}

// ------------------------------------------------------------------ small DFTs (in registers)
// Forward: X_j = sum_q a_q exp(-2 pi i j q / RAD); inverse uses exp(+...).
template <typename R, int RAD> struct Dft;

template <typename R> struct Dft<R, 2> {
  __device__ __forceinline__ static void run(cpx<R>* a, bool) {
    cpx<R> t = a[0] - a[1];
    a[0] = a[0] + a[1];
    a[1] = t;
  }
};

template <typename R> struct Dft<R, 4> {
  __device__ __forceinline__ static void run(cpx<R>* a, bool inv) {
    cpx<R> t0 = a[0] + a[2], t1 = a[0] - a[2], t2 = a[1] + a[3], d = a[1] - a[3];
    cpx<R> t3 = inv ? mul_i(d) : mul_mi(d);
    a[0] = t0 + t2;
    a[2] = t0 - t2;
    a[1] = t1 + t3;
    a[3] = t1 - t3;
  }
};

template <typename R> struct Dft<R, 3> {
  __device__ __forceinline__ static void run(cpx<R>* a, bool inv) {
    const R c = (R)-0.5;
    const R sn = (R)0.86602540378443864676372317075294;  // sin(2 pi / 3)
    cpx<R> s = a[1] + a[2], d = a[1] - a[2];
    cpx<R> m = a[0] + c * s;
    cpx<R> rot = inv ? mul_i(sn * d) : mul_mi(sn * d);
    a[0] = a[0] + s;
    a[1] = m + rot;
    a[2] = m - rot;
  }
};

template <typename R> struct Dft<R, 5> {
  __device__ __forceinline__ static void run(cpx<R>* a, bool inv) {
    const R c1 = (R)0.30901699437494742410229341718282;    // cos(2 pi/5)
    const R c2 = (R)-0.80901699437494742410229341718282;   // cos(4 pi/5)
    const R s1 = (R)0.95105651629515357211643933337938;    // sin(2 pi/5)
    const R s2 = (R)0.58778525229247312916870595463907;    // sin(4 pi/5)
    cpx<R> sa = a[1] + a[4], da = a[1] - a[4], sb = a[2] + a[3], db = a[2] - a[3];
    cpx<R> m1 = a[0] + c1 * sa + c2 * sb;
    cpx<R> m2 = a[0] + c2 * sa + c1 * sb;
    cpx<R> r1 = s1 * da + s2 * db;
    cpx<R> r2 = s2 * da - s1 * db;
    r1 = inv ? mul_i(r1) : mul_mi(r1);
    r2 = inv ? mul_i(r2) : mul_mi(r2);
    a[0] = a[0] + sa + sb;
    a[1] = m1 + r1;
    a[4] = m1 - r1;
    a[2] = m2 + r2;
    a[3] = m2 - r2;
  }
};

// ------------------------------------------------------------------ Stockham pass in smem
// One radix-RAD pass of a self-sorting (Stockham) FFT over `nlines` lines of length n stored
// at buf + line*ld.  p is the product of the radices already applied (1 on the first pass).
// Butterfly b (line l, index i < n/RAD) reads l[i + q n/RAD], q < RAD, multiplies by the
// twiddles exp(-+ 2 pi i q k/(p RAD)) with k = i mod p, applies the RAD-point DFT and writes
// l[(i - k) RAD + k + q p].  After all passes the line holds its DFT in natural order.
// tw[m] = exp(-2 pi i m/n) for m < n (rounded once from FP64).  All reads of the pass finish
// (barrier) before any write, so the pass works in place.  SLOTS*blockDim must cover the
// pass's butterflies.
// Unsigned division by d via a multiply-high with M = ceil(2^32 / d) (the round-up variant of
// Granlund & Montgomery, 1994): floor(x M / 2^32) = floor(x / d) whenever x (M d - 2^32) < 2^32,
// which holds for every x < 2^32 / d; the butterfly indices here stay below 2^16 and d <= 512.
struct FastDiv {
  unsigned d, mag;
  __device__ __forceinline__ explicit FastDiv(unsigned d_) : d(d_), mag(d_ > 1 ? 0xFFFFFFFFu / d_ + 1u : 0u) {}
  __device__ __forceinline__ unsigned div(unsigned x) const { return d > 1 ? __umulhi(x, mag) : x; }
};

template <typename R, int RAD, int SLOTS>
__device__ __forceinline__ void stockham_pass(cpx<R>* buf, int ld, int nlines, int n, int p,
                                              bool inv, const cpx<R>* __restrict__ tw) {
  const int m = n / RAD;
  const int nb = nlines * m;
  const int twstep = n / (p * RAD);
  const FastDiv fm((unsigned)m), fp((unsigned)p);
  cpx<R> v[SLOTS][RAD];
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int b = threadIdx.x + s * blockDim.x;
    if (b < nb) {
      const int line = (int)fm.div((unsigned)b);
      const int i = b - line * m;
      const int k = i - p * (int)fp.div((unsigned)i);
      const cpx<R>* src = buf + line * ld;
#pragma unroll
      for (int q = 0; q < RAD; ++q) v[s][q] = src[i + q * m];
      if (k != 0) {
#pragma unroll
        for (int q = 1; q < RAD; ++q) {
          cpx<R> w = tw[q * k * twstep];
          if (inv) w.y = -w.y;
          v[s][q] = v[s][q] * w;
        }
      }
      Dft<R, RAD>::run(v[s], inv);
    }
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < SLOTS; ++s) {
    const int b = threadIdx.x + s * blockDim.x;
    if (b < nb) {
      const int line = (int)fm.div((unsigned)b);
      const int i = b - line * m;
      const int k = i - p * (int)fp.div((unsigned)i);
      cpx<R>* dst = buf + line * ld + (i - k) * RAD + k;
#pragma unroll
      for (int q = 0; q < RAD; ++q) dst[q * p] = v[s][q];
    }
  }
  __syncthreads();
}

// Radix plan of one axis: radices applied in order (product = n), at most 12 passes.
struct RadixPlan {
  int n;
  int npass;
  int rad[12];
};

// Full in-place FFT of `nlines` lines (forward when !inv).  MAXE bounds the elements a
// thread holds per pass: blockDim * MAXE >= nlines * n + blockDim * 5 must hold.
template <typename R, int MAXE>
__device__ __forceinline__ void fft_lines(cpx<R>* buf, int ld, int nlines, const RadixPlan& pl,
                                          bool inv, const cpx<R>* __restrict__ tw) {
  int p = 1;
  for (int ps = 0; ps < pl.npass; ++ps) {
    const int r = pl.rad[ps];
    if (r == 4) stockham_pass<R, 4, MAXE / 4>(buf, ld, nlines, pl.n, p, inv, tw);
    else if (r == 2) stockham_pass<R, 2, MAXE / 2>(buf, ld, nlines, pl.n, p, inv, tw);
    else if (r == 3) stockham_pass<R, 3, MAXE / 3>(buf, ld, nlines, pl.n, p, inv, tw);
    else stockham_pass<R, 5, MAXE / 5>(buf, ld, nlines, pl.n, p, inv, tw);
    p *= r;
  }
}

}  // namespace swf
