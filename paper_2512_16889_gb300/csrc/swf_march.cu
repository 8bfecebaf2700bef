// Time march of the scattered wave (Sec. II, Eq. 6; Sec. II.A) on the GPU.
//
// Right-hand side, per field f and stage value Y:
//     k = -i [ H0 Y + V(t, x) (Y + psi_b(t, x)) ]
// with H0 applied per Fourier mode (Eq. 10).  One evaluation is a chain of line passes over
// the planar state [f][4][z][y][x]:
//   first pass (x lines):  Y = y + h sum_j a_ij k_j (stage combine, Dormand-Prince), the local
//                          term Z = -i V (Y + psi_b) stashed in the output slot, forward x-FFT;
//   middle passes (y, z):  forward FFT along the axis; on the last axis -i H0(kappa)/N and the
//                          inverse FFT;
//   last pass (x lines):   inverse x-FFT and k = (that) + Z.
// Gauge field and background are analytic and evaluated on the fly from per-field 1D tables
// (every field kind is a product of a time factor and one factor per axis).
#include <array>
#include <atomic>
#include <algorithm>
#include <cmath>
#include <map>
#include <vector>
#include <cstdio>
#include <cstring>

#include "swf_internal.h"

namespace swf {

// ---------------------------------------------------------------- Dormand-Prince 5(4) tableau
// Dormand & Prince (1980); first-same-as-last: the 7th stage value is the new state.
static const double DP_C[7] = {0.0, 1.0 / 5, 3.0 / 10, 4.0 / 5, 8.0 / 9, 1.0, 1.0};
static const double DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5, 0, 0, 0, 0, 0},
    {3.0 / 40, 9.0 / 40, 0, 0, 0, 0},
    {44.0 / 45, -56.0 / 15, 32.0 / 9, 0, 0, 0},
    {19372.0 / 6561, -25360.0 / 2187, 64448.0 / 6561, -212.0 / 729, 0, 0},
    {9017.0 / 3168, -355.0 / 33, 46732.0 / 5247, 49.0 / 176, -5103.0 / 18656, 0},
    {35.0 / 384, 0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84}};

template <typename R>
struct StageArgs {
  cpx<R>* y;
  const cpx<R>* kin[6];
  double coef[6];
  int nterm;
  int write_y;
  cpx<R>* kout;
  cpx<R>* T;
  const FieldDesc* fd;
  const R* greal;       // per field: gx[nx] gy[ny] gz[nz]
  const cpx<R>* gcplx;  // per field: ex[nx] ey[ny] ez[nz] w[4]
  const cpx<R>* tw[3];
  const R* kap;         // mode momenta kappa_j = 2 pi j'/L_a of the axes with n_a > 1, rounded once
                        // from FP64, at offsets 0, nx, nx + ny (FP64 is scarce on this GPU)
  R inv_n;              // 1/N rounded once
  RadixPlan plan[3];
  GridDesc g;
  int nrows;            // ny * nz
  double t;             // stage time when clk is null
  cpx<R>* ystage;       // optional: receives the stage value Y (Breit-Wheeler integrand)
  const struct MarchClock* clk;  // march clock (graph replays), or null
  int ls;               // step within the replayed pair of steps (0 or 1)
  double c;             // Dormand-Prince node c_i of the stage
  const struct StepControl* ctl;  // step-size-controlled march, or null (see march_adaptive)
  cpx<R>* ynew;         // with ctl: the last stage writes the step's result here, not into y
  cpx<R>* yspec;        // optional: receives the grid transform of the stage value (written by the
                        // y or z pass that applies H0, before it does)
  cpx<R>* ylo;          // optional (complex64 fixed-step marches): the rounding error of y, so that
                        // y + ylo carries the state in float-float (Knuth's two-sum per step)
};

// (hi, lo) += s in float-float arithmetic (Knuth's two-sum, then a fast renormalisation): on
// return s holds the new rounded state and lo its rounding error.
__device__ __forceinline__ void ff_accumulate(float hi, float& lo, float& s) {
  const float t = __fadd_rn(hi, s);
  const float bp = __fsub_rn(t, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(s, bp));
  const float l = __fadd_rn(lo, e);
  const float nh = __fadd_rn(t, l);
  lo = __fsub_rn(l, __fsub_rn(nh, t));
  s = nh;
}

// State of a step-size-controlled march, in device memory: the accepted time t and the step h
// of the current attempt (the stage times are t + c_i h and the stage coefficients h a_ij), the
// tolerances, counters and flags.  One thread of k_step_control updates it after every attempt.
struct StepControl {
  double t, h, t_in, span, rtol, atol;
  int done;        // t_in reached, or the march failed: later attempts do nothing
  int ok;          // the last attempt was accepted (its result and k_7 are copied in)
  int failed;      // too many attempts or a non-finite error
  int accepted, rejected, max_attempts;
};

// Device clock of a march whose steps are replayed from a CUDA graph: the stage time is
// (t_out + (step + ls) h) + c_i h, the host loop's arithmetic, with `step` advanced on the device
// after each replay.
struct MarchClock {
  double t_out, h;
  int step;
  int pad;
};

template <typename R>
__device__ __forceinline__ double stage_time(const StageArgs<R>& A) {
  if (A.ctl) return A.ctl->t + A.c * A.ctl->h;
  if (!A.clk) return A.t;
  const double tn = A.clk->t_out + (A.clk->step + A.ls) * A.clk->h;
  return tn + A.c * A.clk->h;
}

__global__ void k_clock_set(MarchClock* c, double t_out, double h) {
  c->t_out = t_out;
  c->h = h;
  c->step = 0;
  c->pad = 0;
}

__global__ void k_clock_advance(MarchClock* c, int by) { c->step += by; }

// ---------------------------------------------------------------- field and background
__device__ __forceinline__ double field_time_factor(const FieldDesc& F, double t, double y) {
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
      if (axis == 1) return F.prm[4] > 0.0 ? exp(-xc * xc / (F.prm[4] * F.prm[4])) : 1.0;
      return 1.0;
    case SWF_FIELD_SINGLE_E:
    case SWF_FIELD_DOUBLE_E: {
      if (axis == 0) {
        if (F.kind == SWF_FIELD_SINGLE_E) return single_e_x(F, xc);
        return single_e_x(F, xc + F.prm[5]) + single_e_x(F, xc - F.prm[5]);
      }
      const double k = F.prm[2 + axis];
      return exp(-(k * xc) * (k * xc));
    }
    default:
      return 0.0;
  }
}

// Per-field tables, computed in FP64 and rounded once to the march precision.
template <typename R>
__global__ void k_tables(const FieldDesc* fd, GridDesc g, R* greal, cpx<R>* gcplx) {
  const int f = blockIdx.y;
  const int nt = g.n[0] + g.n[1] + g.n[2];
  const FieldDesc& F = fd[f];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nt + 4; i += gridDim.x * blockDim.x) {
    if (i < nt) {
      int axis = 0, j = i;
      while (j >= g.n[axis]) { j -= g.n[axis]; ++axis; }
      const double xc = g.n[axis] > 1 ? g.x0[axis] + j * g.dx[axis] : 0.0;
      greal[(size_t)f * nt + i] = (R)axis_factor(F, axis, xc);
      double sn, cs;
      sincos(F.pmom[axis] * xc, &sn, &cs);
      gcplx[(size_t)f * (nt + 4) + i] = mk<R>((R)cs, (R)sn);
    } else {
      const int c = i - nt;
      gcplx[(size_t)f * (nt + 4) + i] = mk<R>((R)F.w[2 * c], (R)F.w[2 * c + 1]);
    }
  }
}

// The mode momenta of every axis, kap[off_a + j] = (R) mode_kappa(j, n_a, L_a) (0 on trivial axes):
// the values the H0 step used to compute per element in FP64.
template <typename R>
__global__ void k_kappa_table(GridDesc g, R* kap) {
  const int nt = g.n[0] + g.n[1] + g.n[2];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nt; i += gridDim.x * blockDim.x) {
    int axis = 0, j = i;
    while (j >= g.n[axis]) { j -= g.n[axis]; ++axis; }
    kap[i] = g.n[axis] > 1 ? (R)mode_kappa(j, g.n[axis], g.L[axis]) : (R)0;
  }
}

// V phi for the one non-zero covariant component A_mu = a (V = A_0 + alpha^k A_k).
template <typename R>
__device__ __forceinline__ void apply_v(int acomp, R a, const cpx<R>* p, cpx<R>* o) {
  switch (acomp) {
    case 0:
      o[0] = a * p[0]; o[1] = a * p[1]; o[2] = a * p[2]; o[3] = a * p[3];
      break;
    case 1:  // alpha^x
      o[0] = a * p[3]; o[1] = a * p[2]; o[2] = a * p[1]; o[3] = a * p[0];
      break;
    case 2:  // alpha^y
      o[0] = a * mul_mi(p[3]); o[1] = a * mul_i(p[2]); o[2] = a * mul_mi(p[1]); o[3] = a * mul_i(p[0]);
      break;
    case 3:  // alpha^z
      o[0] = a * p[2]; o[1] = (R)(-1) * (a * p[3]); o[2] = a * p[0]; o[3] = (R)(-1) * (a * p[1]);
      break;
    default:
      o[0] = o[1] = o[2] = o[3] = mk<R>(0, 0);
  }
}

// v <- -i s (alpha.kappa + beta) v  (Dirac representation, sigma.kappa blocks).
template <typename R>
__device__ __forceinline__ void h0_mi(cpx<R>* v, R kx, R ky, R kz, R s) {
  const cpx<R> a = v[0], b = v[1], c = v[2], d = v[3];
  // sigma.k (u0, u1) = (kz u0 + (kx - i ky) u1, (kx + i ky) u0 - kz u1)
  const cpx<R> sl0 = kz * c + kx * d + ky * mul_mi(d);
  const cpx<R> sl1 = kx * c + ky * mul_i(c) - kz * d;
  const cpx<R> su0 = kz * a + kx * b + ky * mul_mi(b);
  const cpx<R> su1 = kx * a + ky * mul_i(a) - kz * b;
  v[0] = s * mul_mi(a + sl0);
  v[1] = s * mul_mi(b + sl1);
  v[2] = s * mul_mi(su0 - c);
  v[3] = s * mul_mi(su1 - d);
}

__device__ __forceinline__ double kappa_of(int j, int n, double L, double K) {
  return n > 1 ? mode_kappa(j, n, L) : K;
}


// ---------------------------------------------------------------- composite DFTs in registers
// cos and sin of 2 pi e / N for the composite radices (written out to 25 digits).
__host__ __device__ constexpr double tw_const(int N, int e, bool want_cos) {
  if (N == 8) {
    switch (e) {
      case 0: return want_cos ? 1.0000000000000000000000000 : 0.0000000000000000000000000;
      case 1: return want_cos ? 0.7071067811865475244008444 : 0.7071067811865475244008444;
      case 2: return want_cos ? -0.0000000000000000000000000 : 1.0000000000000000000000000;
      case 3: return want_cos ? -0.7071067811865475244008444 : 0.7071067811865475244008444;
      case 4: return want_cos ? -1.0000000000000000000000000 : 0.0000000000000000000000000;
      case 5: return want_cos ? -0.7071067811865475244008444 : -0.7071067811865475244008444;
      case 6: return want_cos ? -0.0000000000000000000000000 : -1.0000000000000000000000000;
      case 7: return want_cos ? 0.7071067811865475244008444 : -0.7071067811865475244008444;
    }
  }
  if (N == 12) {
    switch (e) {
      case 0: return want_cos ? 1.0000000000000000000000000 : 0.0000000000000000000000000;
      case 1: return want_cos ? 0.8660254037844386467637232 : 0.5000000000000000000000000;
      case 2: return want_cos ? 0.5000000000000000000000000 : 0.8660254037844386467637232;
      case 3: return want_cos ? -0.0000000000000000000000000 : 1.0000000000000000000000000;
      case 4: return want_cos ? -0.5000000000000000000000000 : 0.8660254037844386467637232;
      case 5: return want_cos ? -0.8660254037844386467637232 : 0.5000000000000000000000000;
      case 6: return want_cos ? -1.0000000000000000000000000 : 0.0000000000000000000000000;
      case 7: return want_cos ? -0.8660254037844386467637232 : -0.5000000000000000000000000;
      case 8: return want_cos ? -0.5000000000000000000000000 : -0.8660254037844386467637232;
      case 9: return want_cos ? -0.0000000000000000000000000 : -1.0000000000000000000000000;
      case 10: return want_cos ? 0.5000000000000000000000000 : -0.8660254037844386467637232;
      case 11: return want_cos ? 0.8660254037844386467637232 : -0.5000000000000000000000000;
    }
  }
  if (N == 16) {
    switch (e) {
      case 0: return want_cos ? 1.0000000000000000000000000 : 0.0000000000000000000000000;
      case 1: return want_cos ? 0.9238795325112867561281832 : 0.3826834323650897717284600;
      case 2: return want_cos ? 0.7071067811865475244008444 : 0.7071067811865475244008444;
      case 3: return want_cos ? 0.3826834323650897717284600 : 0.9238795325112867561281832;
      case 4: return want_cos ? -0.0000000000000000000000000 : 1.0000000000000000000000000;
      case 5: return want_cos ? -0.3826834323650897717284600 : 0.9238795325112867561281832;
      case 6: return want_cos ? -0.7071067811865475244008444 : 0.7071067811865475244008444;
      case 7: return want_cos ? -0.9238795325112867561281832 : 0.3826834323650897717284600;
      case 8: return want_cos ? -1.0000000000000000000000000 : 0.0000000000000000000000000;
      case 9: return want_cos ? -0.9238795325112867561281832 : -0.3826834323650897717284600;
      case 10: return want_cos ? -0.7071067811865475244008444 : -0.7071067811865475244008444;
      case 11: return want_cos ? -0.3826834323650897717284600 : -0.9238795325112867561281832;
      case 12: return want_cos ? -0.0000000000000000000000000 : -1.0000000000000000000000000;
      case 13: return want_cos ? 0.3826834323650897717284600 : -0.9238795325112867561281832;
      case 14: return want_cos ? 0.7071067811865475244008444 : -0.7071067811865475244008444;
      case 15: return want_cos ? 0.9238795325112867561281832 : -0.3826834323650897717284600;
    }
  }
  if (N == 20) {
    switch (e) {
      case 0: return want_cos ? 1.0000000000000000000000000 : 0.0000000000000000000000000;
      case 1: return want_cos ? 0.9510565162951535721164393 : 0.3090169943749474241022934;
      case 2: return want_cos ? 0.8090169943749474241022934 : 0.5877852522924731291687060;
      case 3: return want_cos ? 0.5877852522924731291687060 : 0.8090169943749474241022934;
      case 4: return want_cos ? 0.3090169943749474241022934 : 0.9510565162951535721164393;
      case 5: return want_cos ? -0.0000000000000000000000000 : 1.0000000000000000000000000;
      case 6: return want_cos ? -0.3090169943749474241022934 : 0.9510565162951535721164393;
      case 7: return want_cos ? -0.5877852522924731291687060 : 0.8090169943749474241022934;
      case 8: return want_cos ? -0.8090169943749474241022934 : 0.5877852522924731291687060;
      case 9: return want_cos ? -0.9510565162951535721164393 : 0.3090169943749474241022934;
      case 10: return want_cos ? -1.0000000000000000000000000 : 0.0000000000000000000000000;
      case 11: return want_cos ? -0.9510565162951535721164393 : -0.3090169943749474241022934;
      case 12: return want_cos ? -0.8090169943749474241022934 : -0.5877852522924731291687060;
      case 13: return want_cos ? -0.5877852522924731291687060 : -0.8090169943749474241022934;
      case 14: return want_cos ? -0.3090169943749474241022934 : -0.9510565162951535721164393;
      case 15: return want_cos ? -0.0000000000000000000000000 : -1.0000000000000000000000000;
      case 16: return want_cos ? 0.3090169943749474241022934 : -0.9510565162951535721164393;
      case 17: return want_cos ? 0.5877852522924731291687060 : -0.8090169943749474241022934;
      case 18: return want_cos ? 0.8090169943749474241022934 : -0.5877852522924731291687060;
      case 19: return want_cos ? 0.9510565162951535721164393 : -0.3090169943749474241022934;
    }
  }
  return 0.0;
}

// v * W_N^e (forward, W = exp(-2 pi i / N)) or v * conj(W_N^e) (inverse); quarter turns exact.
template <typename R>
__device__ __forceinline__ cpx<R> twiddle_const(cpx<R> v, int N, int e, bool inv) {
  if (e == 0) return v;
  if ((4 * e) % N == 0) {
    const int q = (4 * e / N) & 3;
    if (q == 2) return mk<R>(-v.x, -v.y);
    if ((q == 1) != inv) return mul_mi(v);
    return mul_i(v);
  }
  const R c = (R)tw_const(N, e, true), s = (R)tw_const(N, e, false);
  return v * mk<R>(c, inv ? s : -s);
}

// DFT of length A*B in registers (Cooley-Tukey): index n = B n1 + n2 in, k = k1 + A k2 out.
template <typename R, int A, int B>
struct DftCT {
  __device__ __forceinline__ static void run(cpx<R>* a, bool inv) {
    constexpr int N = A * B;
    cpx<R> y[N];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) {
      cpx<R> t[A];
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) t[n1] = a[B * n1 + n2];
      Dft<R, A>::run(t, inv);
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) y[n2 * A + k1] = twiddle_const<R>(t[k1], N, n2 * k1, inv);
    }
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) {
      cpx<R> t[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) t[n2] = y[n2 * A + k1];
      Dft<R, B>::run(t, inv);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) a[k1 + A * k2] = t[k2];
    }
  }
};
template <typename R> struct Dft<R, 8> : DftCT<R, 4, 2> {};
template <typename R> struct Dft<R, 12> : DftCT<R, 4, 3> {};
template <typename R> struct Dft<R, 16> : DftCT<R, 4, 4> {};
template <typename R> struct Dft<R, 20> : DftCT<R, 4, 5> {};

// ---------------------------------------------------------------- out-of-place line FFT
// Element e of a line sits at e + e/32 (a gap every 32 elements spreads the strided stores of
// the early passes over the shared-memory banks).
__host__ __device__ __forceinline__ int pad32(int e) { return e + (e >> 5); }
static inline int padded_len(int n) { return pad32(n - 1) + 1; }

// One self-sorting (Stockham) radix-RAD pass from `src` to `dst` over `nlines` lines of length
// n (stride ld, padded positions): butterfly (line, i < n/RAD) reads elements i + q n/RAD,
// multiplies by exp(-+ 2 pi i q k/(p RAD)) (k = i mod p, p = product of the radices so far),
// applies the RAD-point DFT and writes elements (i - k) RAD + k + q p.  Out of place, so each
// butterfly finishes before the next starts (one barrier per pass).
template <typename R, int RAD>
__device__ __forceinline__ void pp_pass(const cpx<R>* __restrict__ src, cpx<R>* __restrict__ dst, int ld,
                                        int nlines, int n, int p, bool inv, const cpx<R>* __restrict__ tw) {
  const int m = n / RAD;
  const int nb = nlines * m;
  const int twstep = n / (p * RAD);
  const FastDiv fm((unsigned)m), fp((unsigned)p);
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const int line = (int)fm.div((unsigned)b);
    const int i = b - line * m;
    const int k = i - p * (int)fp.div((unsigned)i);
    const cpx<R>* s = src + line * ld;
    cpx<R>* d = dst + line * ld;
    cpx<R> v[RAD];
#pragma unroll
    for (int q = 0; q < RAD; ++q) v[q] = s[pad32(i + q * m)];
    if (k != 0) {
      const int ks = k * twstep;
      if (RAD <= 5) {
#pragma unroll
        for (int q = 1; q < RAD; ++q) {
          cpx<R> w = tw[q * ks];
          if (inv) w.y = -w.y;
          v[q] = v[q] * w;
        }
      } else {
        // w^q for q < RAD from the table entries at the powers of two (at most three products
        // per factor: a few units in the last place)
        cpx<R> w[RAD];
#pragma unroll
        for (int q = 1; q < RAD; ++q) {
          if ((q & (q - 1)) == 0) {
            w[q] = tw[q * ks];
            if (inv) w[q].y = -w[q].y;
          } else {
            const int lo = q & (-q);  // lowest set bit: w^q = w^lo w^(q - lo)
            w[q] = w[lo] * w[q - lo];
          }
          v[q] = v[q] * w[q];
        }
      }
    }
    Dft<R, RAD>::run(v, inv);
    const int o = (i - k) * RAD + k;
#pragma unroll
    for (int q = 0; q < RAD; ++q) d[pad32(o + q * p)] = v[q];
  }
  __syncthreads();
}

// Full FFT of `nlines` lines held in `a` (padded layout; the caller has synchronised after
// writing them), using `b` as the second buffer.  Returns the buffer holding the result.
template <typename R>
__device__ cpx<R>* fft_pp(cpx<R>* a, cpx<R>* b, int ld, int nlines, const RadixPlan& pl, bool inv,
                          const cpx<R>* __restrict__ tw) {
  int p = 1;
  for (int ps = 0; ps < pl.npass; ++ps) {
    const int r = pl.rad[ps];
    switch (r) {
      case 16: pp_pass<R, 16>(a, b, ld, nlines, pl.n, p, inv, tw); break;
      case 20: pp_pass<R, 20>(a, b, ld, nlines, pl.n, p, inv, tw); break;
      case 12: pp_pass<R, 12>(a, b, ld, nlines, pl.n, p, inv, tw); break;
      case 8: pp_pass<R, 8>(a, b, ld, nlines, pl.n, p, inv, tw); break;
      case 4: pp_pass<R, 4>(a, b, ld, nlines, pl.n, p, inv, tw); break;
      case 2: pp_pass<R, 2>(a, b, ld, nlines, pl.n, p, inv, tw); break;
      case 3: pp_pass<R, 3>(a, b, ld, nlines, pl.n, p, inv, tw); break;
      default: pp_pass<R, 5>(a, b, ld, nlines, pl.n, p, inv, tw); break;
    }
    cpx<R>* t = a;
    a = b;
    b = t;
    p *= r;
  }
  return a;
}

// ---------------------------------------------------------------- pass kernels
// Shared memory of every pass kernel: two line buffers (the FFT works out of place) within
// kPassSmem, so that three blocks of 256 threads fit an SM.
static const size_t kPassSmem = 72 * 1024;
// The tuner may also try wider shapes (more rows per x block, wider y/z tiles) up to this much
// shared memory per block (one or two blocks per SM): wider y/z tiles read longer contiguous
// runs of each line and give every FFT pass more butterflies per barrier.
static const size_t kPassSmemTune = 200 * 1024;

// x lines of `rows` grid rows (4 components each): stage combine, local term, forward x-FFT
// (and the whole derivative when x is the only non-trivial axis).
// Block (bx, f) of the pass: rows bx*rows .. of field f.
template <typename R>
__device__ __forceinline__ void first_body(const StageArgs<R>& A, int bx, int f, int rows, int ld, int only_x) {
  if (A.ctl && A.ctl->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* buf = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* buf2 = buf + 4 * rows * ld;
  const double hscale = A.ctl ? A.ctl->h : 1.0;  // stage coefficients are a_ij (times h here) under control
  cpx<R>* const yout = A.ynew ? A.ynew : A.y;
  __shared__ R s_ft[64];  // field time factor per row, computed in FP64 and rounded once
  __shared__ cpx<R> s_tf;
  const int row0 = bx * rows;
  const int nx = A.g.n[0], ny = A.g.n[1], nz = A.g.n[2];
  const int N = A.g.N;
  const size_t fo = (size_t)f * 4 * N;
  const FieldDesc* F = A.fd + f;
  const double tst = stage_time(A);
  for (int j = threadIdx.x; j < rows; j += blockDim.x) {
    const int iy = (row0 + j) % ny;
    const double yc = ny > 1 ? A.g.x0[1] + iy * A.g.dx[1] : 0.0;
    s_ft[j] = (R)field_time_factor(*F, tst, yc);
  }
  if (threadIdx.x == 0) {
    double sn, cs;
    sincos(F->tsign * F->e0 * tst, &sn, &cs);
    s_tf = mk<R>((R)cs, (R)sn);
  }
  __syncthreads();
  const int nt = nx + ny + nz;
  const R* gx = A.greal + (size_t)f * nt;
  const R* gy = gx + nx;
  const R* gz = gy + ny;
  const cpx<R>* ex = A.gcplx + (size_t)f * (nt + 4);
  const cpx<R>* ey = ex + nx;
  const cpx<R>* ez = ey + ny;
  const cpx<R>* wsp = ez + nz;
  const int acomp = F->acomp;
  const int per = rows * nx;
  const size_t cs = (size_t)N;
  for (int e = threadIdx.x; e < per; e += blockDim.x) {
    const int j = e / nx;
    const int x = e - j * nx;
    const int row = row0 + j;
    cpx<R> v[4];
    if (row < A.nrows) {
      const size_t gi = fo + (size_t)row * nx + x;
      if (sizeof(R) == 4 && A.ylo && A.write_y) {
        // the new state: the step's increment h sum_j b_j k_j apart, then (y, ylo) += it in
        // float-float, so that the single-precision rounding of y does not accumulate over steps
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = mk<R>(0, 0);
#pragma unroll
        for (int q = 0; q < 6; ++q)
          if (q < A.nterm) {
            const R co = (R)(A.coef[q] * hscale);
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] = v[c] + co * A.kin[q][gi + c * cs];
          }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const cpx<R> yh = A.y[gi + c * cs];
          cpx<R> lo = A.ylo[gi + c * cs];
          float sx = (float)v[c].x, sy = (float)v[c].y, lx = (float)lo.x, ly = (float)lo.y;
          ff_accumulate((float)yh.x, lx, sx);
          ff_accumulate((float)yh.y, ly, sy);
          v[c] = mk<R>((R)sx, (R)sy);
          A.ylo[gi + c * cs] = mk<R>((R)lx, (R)ly);
        }
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = A.y[gi + c * cs];
#pragma unroll
        for (int q = 0; q < 6; ++q)
          if (q < A.nterm) {
            const R co = (R)(A.coef[q] * hscale);
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] = v[c] + co * A.kin[q][gi + c * cs];
          }
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        if (A.write_y) yout[gi + c * cs] = v[c];
        if (A.ystage) A.ystage[gi + c * cs] = v[c];
      }
      // local term Z = -i V (Y + psi_b), kept in the output slot until the last pass
      const int iy = row % ny, iz = row / ny;
      const R a = s_ft[j] * gx[x] * gy[iy] * gz[iz];
      const cpx<R> ph = s_tf * ex[x] * ey[iy] * ez[iz];
      cpx<R> phi[4], vz[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) phi[c] = v[c] + wsp[c] * ph;
      apply_v<R>(acomp, a, phi, vz);
#pragma unroll
      for (int c = 0; c < 4; ++c) A.kout[gi + c * cs] = mul_mi(vz[c]);
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) v[c] = mk<R>(0, 0);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) buf[(c * rows + j) * ld + pad32(x)] = v[c];
  }
  __syncthreads();
  cpx<R>* res = fft_pp<R>(buf, buf2, ld, 4 * rows, A.plan[0], false, A.tw[0]);
  if (!only_x) {
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int j = e / nx;
      const int x = e - j * nx;
      const int row = row0 + j;
      if (row < A.nrows) {
        const size_t gi = fo + (size_t)row * nx + x;
#pragma unroll
        for (int c = 0; c < 4; ++c) A.T[gi + c * cs] = res[(c * rows + j) * ld + pad32(x)];
      }
    }
    return;
  }
  // one non-trivial axis: the whole derivative in this block
  const R sc = A.inv_n;
  const R kx0 = (R)F->K[0], ky = (R)F->K[1], kz = (R)F->K[2];
  for (int e = threadIdx.x; e < per; e += blockDim.x) {
    const int j = e / nx, x = e - j * nx;
    cpx<R> v[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = res[(c * rows + j) * ld + pad32(x)];
    h0_mi<R>(v, nx > 1 ? A.kap[x] : kx0, ky, kz, sc);
#pragma unroll
    for (int c = 0; c < 4; ++c) res[(c * rows + j) * ld + pad32(x)] = v[c];
  }
  __syncthreads();
  res = fft_pp<R>(res, res == buf ? buf2 : buf, ld, 4 * rows, A.plan[0], true, A.tw[0]);
  for (int e = threadIdx.x; e < per; e += blockDim.x) {
    const int j = e / nx;
    const int x = e - j * nx;
    const int row = row0 + j;
    if (row < A.nrows) {
      const size_t gi = fo + (size_t)row * nx + x;
#pragma unroll
      for (int c = 0; c < 4; ++c) A.kout[gi + c * cs] = A.kout[gi + c * cs] + res[(c * rows + j) * ld + pad32(x)];
    }
  }
}

// The x-pass kernels are held to 64 registers in complex64 (no spills), so that four 256-thread
// blocks fit an SM when the tuner picks a shape of at most 56 KB of shared memory.
template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2) k_first(StageArgs<R> A, int rows, int ld, int only_x) {
  first_body<R>(A, blockIdx.x, blockIdx.y, rows, ld, only_x);
}

// Lines along axis 1 (y) or 2 (z) of a tile of TX = 2^lgtx consecutive x columns: forward FFT,
// -i H0(kappa)/N, inverse FFT, as selected.  The tile sits in shared memory as 4 TX lines of
// stride ld (chosen so that the transposing loads and stores of a warp spread over the banks).
// Block (bx, f): tile bx of field f.
template <typename R>
__device__ __forceinline__ void mid_body(const StageArgs<R>& A, int bx, int f, int axis, int lgtx, int ld, int do_fwd,
                                         int do_h0, int do_inv) {
  if (A.ctl && A.ctl->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* buf = reinterpret_cast<cpx<R>*>(smem_raw);
  const int nx = A.g.n[0], ny = A.g.n[1], nz = A.g.n[2];
  const int N = A.g.N;
  const int na = A.g.n[axis];
  const int TX = 1 << lgtx;
  cpx<R>* buf2 = buf + 4 * TX * ld;
  const int ntx = (nx + TX - 1) >> lgtx;
  const int xt = bx % ntx;
  const int o = bx / ntx;  // z index (axis 1) or y index (axis 2)
  const size_t base = axis == 1 ? (size_t)o * nx * ny : (size_t)o * nx;
  const size_t stride = axis == 1 ? (size_t)nx : (size_t)nx * ny;
  const size_t fo = (size_t)f * 4 * N;
  const size_t cs = (size_t)N;
  const int per = TX * na;
  for (int e = threadIdx.x; e < per; e += blockDim.x) {
    const int m = e >> lgtx;
    const int t = e & (TX - 1);
    const int x = xt * TX + t;
    const size_t gi = fo + base + m * stride + x;
#pragma unroll
    for (int c = 0; c < 4; ++c) buf[(c * TX + t) * ld + pad32(m)] = x < nx ? A.T[gi + c * cs] : mk<R>(0, 0);
  }
  __syncthreads();
  cpx<R>* res = buf;
  if (do_fwd) res = fft_pp<R>(res, buf2, ld, 4 * TX, A.plan[axis], false, A.tw[axis]);
  if (do_h0 && A.yspec) {
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int m = e >> lgtx;
      const int t = e & (TX - 1);
      const int x = xt * TX + t;
      if (x < nx) {
        const size_t gi = fo + base + m * stride + x;
#pragma unroll
        for (int c = 0; c < 4; ++c) A.yspec[gi + c * cs] = res[(c * TX + t) * ld + pad32(m)];
      }
    }
    __syncthreads();
  }
  if (do_h0) {
    const FieldDesc* F = A.fd + f;
    const R sc = A.inv_n;
    const R K0 = (R)F->K[0], K1 = (R)F->K[1], K2 = (R)F->K[2];  // momenta along trivial axes
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int t = e / na, m = e - t * na;
      const int x = xt * TX + t;
      if (x >= nx) continue;
      const int iy = axis == 1 ? m : o;
      const int iz = axis == 2 ? m : o;
      cpx<R> v[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) v[c] = res[(c * TX + t) * ld + pad32(m)];
      h0_mi<R>(v, nx > 1 ? A.kap[x] : K0, ny > 1 ? A.kap[nx + iy] : K1, nz > 1 ? A.kap[nx + ny + iz] : K2, sc);
#pragma unroll
      for (int c = 0; c < 4; ++c) res[(c * TX + t) * ld + pad32(m)] = v[c];
    }
    __syncthreads();
  }
  if (do_inv) res = fft_pp<R>(res, res == buf ? buf2 : buf, ld, 4 * TX, A.plan[axis], true, A.tw[axis]);
  for (int e = threadIdx.x; e < per; e += blockDim.x) {
    const int m = e >> lgtx;
    const int t = e & (TX - 1);
    const int x = xt * TX + t;
    if (x < nx) {
      const size_t gi = fo + base + m * stride + x;
#pragma unroll
      for (int c = 0; c < 4; ++c) A.T[gi + c * cs] = res[(c * TX + t) * ld + pad32(m)];
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(256) k_mid(StageArgs<R> A, int axis, int lgtx, int ld, int do_fwd, int do_h0,
                                             int do_inv) {
  mid_body<R>(A, blockIdx.x, blockIdx.y, axis, lgtx, ld, do_fwd, do_h0, do_inv);
}

// x lines: inverse x-FFT, k = (that) + Z.  Block (bx, f): rows bx*rows .. of field f.
template <typename R>
__device__ __forceinline__ void last_body(const StageArgs<R>& A, int bx, int f, int rows, int ld) {
  if (A.ctl && A.ctl->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* buf = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* buf2 = buf + 4 * rows * ld;
  const int row0 = bx * rows;
  const int nx = A.g.n[0];
  const int N = A.g.N;
  const size_t fo = (size_t)f * 4 * N;
  const size_t cs = (size_t)N;
  const int per = rows * nx;
  for (int e = threadIdx.x; e < per; e += blockDim.x) {
    const int j = e / nx;
    const int x = e - j * nx;
    const int row = row0 + j;
    const size_t gi = fo + (size_t)row * nx + x;
#pragma unroll
    for (int c = 0; c < 4; ++c)
      buf[(c * rows + j) * ld + pad32(x)] = row < A.nrows ? A.T[gi + c * cs] : mk<R>(0, 0);
  }
  __syncthreads();
  cpx<R>* res = fft_pp<R>(buf, buf2, ld, 4 * rows, A.plan[0], true, A.tw[0]);
  for (int e = threadIdx.x; e < per; e += blockDim.x) {
    const int j = e / nx;
    const int x = e - j * nx;
    const int row = row0 + j;
    if (row < A.nrows) {
      const size_t gi = fo + (size_t)row * nx + x;
#pragma unroll
      for (int c = 0; c < 4; ++c) A.kout[gi + c * cs] = A.kout[gi + c * cs] + res[(c * rows + j) * ld + pad32(x)];
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2) k_last(StageArgs<R> A, int rows, int ld) {
  last_body<R>(A, blockIdx.x, blockIdx.y, rows, ld);
}

// The x lines of one evaluation's end and the next one's start in one launch: k_i = inverse
// x-FFT of T + Z for stage P, then the stage combine, local term and forward x-FFT of stage Nx on
// the same rows.  Each thread reads back the k_i entries it has just written (the two bodies map
// the rows' entries to threads alike), so the arithmetic is that of k_last then k_first.
template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 4 : 2) k_last_first(StageArgs<R> P, StageArgs<R> Nx, int rows, int ld) {
  last_body<R>(P, blockIdx.x, blockIdx.y, rows, ld);
  __syncthreads();
  first_body<R>(Nx, blockIdx.x, blockIdx.y, rows, ld, 0);
}

// ---------------------------------------------------------------- host side
template <typename R> struct Prec;
template <> struct Prec<float> { static constexpr int is_double = 0; };
template <> struct Prec<double> { static constexpr int is_double = 1; };

static const int kThreads = 256;

// Radix plan of the march's line FFTs: radix 16 first, then the composite radices 20 and 12,
// then 8, 4, 2, 3, 5 (every length of the form 2^a 3^b 5^c).
static bool make_march_plan(int n, RadixPlan* pl) {
  pl->n = n;
  pl->npass = 0;
  int m = n;
  const int order[8] = {16, 20, 12, 8, 4, 2, 3, 5};
  for (int r : order)
    while (m % r == 0 && pl->npass < 12) {
      pl->rad[pl->npass++] = r;
      m /= r;
    }
  return m == 1;
}

// Streaming multiprocessors of the current device (cached per device).
static int sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
  if (cache[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
    cache[dev] = n;
  }
  return cache[dev];
}

// Rows per block of the x passes: as many as fit kPassSmem (at most 64), fewer on small grids
// (up to two blocks per SM).  0 if one row does not fit.
template <typename R>
static int x_rows(int nx, int nrows, int F) {
  const size_t line = (size_t)2 * 4 * padded_len(nx) * sizeof(cpx<R>);
  int rows = (int)(kPassSmem / line);
  if (rows > 64) rows = 64;
  if (rows > nrows) rows = nrows;
  while (rows > 1 && (long)F * ((nrows + rows - 1) / rows) < 2L * sm_count()) rows = (rows + 1) / 2;
  return rows;
}

// Tile of a y or z pass: the widest power-of-two column count TX <= 16 whose two buffers fit
// kPassSmem, narrowed on small grids (down to 32 bytes of contiguous x per line) for up to two
// blocks per SM; line stride ld >= the padded length with ld = 32/TX modulo the elements of one
// 128-byte shared-memory wavefront, so that the transposing accesses of a warp (TX columns x
// 32/TX lines) fall on distinct banks.  `tiles` = (field, other-axis index) pairs of the pass.
struct MidShape {
  int lgtx, ld;
  size_t smem;
};

template <typename R>
static int mid_stride(int n_a, int lg) {
  const int unit = 128 / (int)sizeof(cpx<R>);
  const int base = padded_len(n_a);
  const int pad = (((32 >> lg) % unit - base % unit) % unit + unit) % unit;
  return base + pad;
}

template <typename R>
static size_t mid_smem(int n_a, int lg) {
  return (size_t)2 * 4 * (1 << lg) * mid_stride<R>(n_a, lg) * sizeof(cpx<R>);
}

// widest tile that fits `cap` bytes of shared memory (TX <= nx as well)
template <typename R>
static int mid_max_lg(int n_a, int nx, size_t cap = kPassSmem) {
  int lg = 4;
  while (lg > 0 && ((1 << lg) > nx || mid_smem<R>(n_a, lg) > cap)) --lg;
  return lg;
}

template <typename R>
static MidShape mid_shape_lg(int n_a, int lg) {
  MidShape m{};
  m.lgtx = lg;
  m.ld = mid_stride<R>(n_a, lg);
  m.smem = mid_smem<R>(n_a, lg);
  return m;
}

template <typename R>
static MidShape mid_shape(int n_a, int nx, long tiles) {
  const int min_lg = sizeof(cpx<R>) == 8 ? 2 : 1;
  int lg = mid_max_lg<R>(n_a, nx);
  while (lg > min_lg && tiles * ((nx + (1 << lg) - 1) >> lg) < 2L * sm_count()) --lg;
  return mid_shape_lg<R>(n_a, lg);
}

// Keys of the tuned shapes: pass kind, element size and the sizes that decide the launch.
static std::string tune_key(char kind, int esz, int a, int b, int c, long d) {
  char buf[96];
  std::snprintf(buf, sizeof buf, "%c/%d/%d/%d/%d/%ld", kind, esz, a, b, c, d);
  return buf;
}

static int tune_lookup(swf_ctx* ctx, const std::string& key, int fallback) {
  if (!ctx || !ctx->tune.on) return fallback;
  auto it = ctx->tune.best.find(key);
  return it == ctx->tune.best.end() ? fallback : it->second;
}

template <typename R>
static swf_status set_smem_attrs() {
  // per device; several host threads may arrive at once, and setting the attributes twice is harmless
  static std::atomic<bool> done[64];
  const int dv = dev_slot();
  if (done[dv].load(std::memory_order_acquire)) return SWF_OK;
  cudaError_t e;
  e = cudaFuncSetAttribute(k_first<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmemTune);
  if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(k_first)");
  e = cudaFuncSetAttribute(k_mid<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmemTune);
  if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(k_mid)");
  e = cudaFuncSetAttribute(k_last<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmemTune);
  if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(k_last)");
  e = cudaFuncSetAttribute(k_last_first<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmemTune);
  if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(k_last_first)");
  done[dv].store(true, std::memory_order_release);
  return SWF_OK;
}

// Launch shape of the x passes (k_first, k_last, k_last_first): rows per block, threads, padded
// line length, shared memory, grid.
struct XLaunch {
  int rows, thr, ld;
  size_t smem;
  dim3 grid;
};

template <typename R>
static XLaunch x_launch(swf_ctx* ctx, const StageArgs<R>& A, int F) {
  constexpr int esz = (int)sizeof(cpx<R>);
  const int nx = A.g.n[0];
  // tuned values: rows (x passes) or log2 TX (y, z passes) times 4, plus 1 for 128-thread blocks
  const int xv = tune_lookup(ctx, tune_key('x', esz, nx, A.nrows, 0, F), 4 * x_rows<R>(nx, A.nrows, F));
  XLaunch L;
  L.rows = xv >> 2;
  L.thr = (xv & 3) ? kThreads / 2 : kThreads;
  L.ld = padded_len(nx);
  L.smem = (size_t)2 * 4 * (L.rows > 0 ? L.rows : 1) * L.ld * sizeof(cpx<R>);
  L.grid = dim3(L.rows > 0 ? (A.nrows + L.rows - 1) / L.rows : 1, F);
  return L;
}

// The y and z passes of one evaluation.
template <typename R>
static void launch_mids(swf_ctx* ctx, const StageArgs<R>& A, int F, cudaStream_t st) {
  const int nx = A.g.n[0], ny = A.g.n[1], nz = A.g.n[2];
  constexpr int esz = (int)sizeof(cpx<R>);
  int axes[2], na = 0;
  if (ny > 1) axes[na++] = 1;
  if (nz > 1) axes[na++] = 2;
  auto mid = [&](int axis, int fwd, int h0, int inv) {
    const int other = axis == 1 ? nz : ny;
    const int lg_h = mid_shape<R>(A.g.n[axis], nx, (long)other * F).lgtx;
    const int mv = tune_lookup(ctx, tune_key('m', esz, axis * 8 + fwd * 4 + h0 * 2 + inv, A.g.n[axis], nx, (long)other * F),
                               4 * lg_h);
    const MidShape ms = mid_shape_lg<R>(A.g.n[axis], mv >> 2);
    const int ntx = (nx + (1 << ms.lgtx) - 1) >> ms.lgtx;
    dim3 grid(ntx * other, F);
    ProfScope ps(ctx, "k_mid", st);
    k_mid<R><<<grid, (mv & 3) ? kThreads / 2 : kThreads, ms.smem, st>>>(A, axis, ms.lgtx, ms.ld, fwd, h0, inv);
  };
  if (na == 1) {
    mid(axes[0], 1, 1, 1);
  } else if (na == 2) {
    mid(1, 1, 0, 0);
    mid(2, 1, 1, 1);
    mid(1, 0, 0, 1);
  }
}

// Launches one right-hand-side evaluation for F fields (ctx may be null: no profiling).
template <typename R>
static swf_status launch_eval(swf_ctx* ctx, const StageArgs<R>& A, int F, cudaStream_t st) {
  const bool only_x = (A.g.n[1] == 1 && A.g.n[2] == 1);
  const XLaunch L = x_launch<R>(ctx, A, F);
  if (L.rows < 1) return SWF_EUNSUPPORTED;
  {
    ProfScope ps(ctx, "k_first", st);
    k_first<R><<<L.grid, L.thr, L.smem, st>>>(A, L.rows, L.ld, only_x ? 1 : 0);
  }
  if (only_x) return SWF_OK;
  launch_mids<R>(ctx, A, F, st);
  {
    ProfScope ps(ctx, "k_last", st);
    k_last<R><<<L.grid, L.thr, L.smem, st>>>(A, L.rows, L.ld);
  }
  return SWF_OK;
}

// An evaluation whose inverse x pass is left for the next launch (march chains with at least one
// non-trivial axis besides x): k_first and the y/z passes of A.
template <typename R>
static swf_status launch_eval_open(swf_ctx* ctx, const StageArgs<R>& A, int F, cudaStream_t st) {
  const XLaunch L = x_launch<R>(ctx, A, F);
  if (L.rows < 1) return SWF_EUNSUPPORTED;
  {
    ProfScope ps(ctx, "k_first", st);
    k_first<R><<<L.grid, L.thr, L.smem, st>>>(A, L.rows, L.ld, 0);
  }
  launch_mids<R>(ctx, A, F, st);
  return SWF_OK;
}

// Closes the open evaluation P and runs evaluation Nx with it: k_last_first, then Nx's y/z passes.
template <typename R>
static swf_status launch_eval_chain(swf_ctx* ctx, const StageArgs<R>& P, const StageArgs<R>& Nx, int F,
                                    cudaStream_t st) {
  const XLaunch L = x_launch<R>(ctx, Nx, F);
  if (L.rows < 1) return SWF_EUNSUPPORTED;
  {
    ProfScope ps(ctx, "k_last_first", st);
    k_last_first<R><<<L.grid, L.thr, L.smem, st>>>(P, Nx, L.rows, L.ld);
  }
  launch_mids<R>(ctx, Nx, F, st);
  return SWF_OK;
}

// Closes the open evaluation P (its inverse x pass).
template <typename R>
static swf_status launch_eval_close(swf_ctx* ctx, const StageArgs<R>& P, int F, cudaStream_t st) {
  const XLaunch L = x_launch<R>(ctx, P, F);
  if (L.rows < 1) return SWF_EUNSUPPORTED;
  ProfScope ps(ctx, "k_last", st);
  k_last<R><<<L.grid, L.thr, L.smem, st>>>(P, L.rows, L.ld);
  return SWF_OK;
}

// Times the candidate launch shapes of one evaluation's pass kernels (rows per block or tile
// width, and 256- or 128-thread blocks) and records the fastest in ctx->tune (once per shape key).  B must be harmless to run repeatedly: it may write only
// T and its output slot, and read y and its input slots (the march calls this before its first
// evaluation, when those hold nothing yet).  The shape decides only which lines a block
// transforms, never the arithmetic of a line, so results do not depend on the choice.
template <typename R>
static swf_status autotune_eval(swf_ctx* ctx, const StageArgs<R>& B, int F, cudaStream_t st) {
  if (!ctx || !ctx->tune.on) return SWF_OK;
  constexpr int esz = (int)sizeof(cpx<R>);
  const int nx = B.g.n[0], ny = B.g.n[1], nz = B.g.n[2];
  const bool only_x = (ny == 1 && nz == 1);
  cudaEvent_t ev[2];
  if (cudaEventCreate(&ev[0]) != cudaSuccess) return cuda_status(cudaGetLastError(), "tuning events");
  if (cudaEventCreate(&ev[1]) != cudaSuccess) {
    cudaEventDestroy(ev[0]);
    return cuda_status(cudaGetLastError(), "tuning events");
  }
  swf_status status = SWF_OK;
  // time `launch` (one warm-up, then three back to back); +inf on a launch error
  auto timed = [&](auto&& launch) -> float {
    launch();
    cudaEventRecord(ev[0], st);
    for (int r = 0; r < 3; ++r) launch();
    cudaEventRecord(ev[1], st);
    cudaError_t e = cudaEventSynchronize(ev[1]);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) {
      status = cuda_status(e, "tuning launches");
      return 3.4e38f;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev[0], ev[1]);
    return ms;
  };
  const std::string xkey = tune_key('x', esz, nx, B.nrows, 0, F);
  if (!ctx->tune.best.count(xkey)) {
    const size_t line = (size_t)2 * 4 * padded_len(nx) * esz;
    int rmax = (int)(kPassSmemTune / line);
    rmax = std::min(std::min(rmax, 64), B.nrows);
    int best = 4 * x_rows<R>(nx, B.nrows, F);
    float tbest = 3.4e38f;
    const int ld = padded_len(nx);
    for (int rows = 1; rows <= rmax && status == SWF_OK; rows *= 2) {
      for (int half = 0; half < 2 && status == SWF_OK; ++half) {
        const int thr = half ? kThreads / 2 : kThreads;
        const size_t smem = (size_t)2 * 4 * rows * ld * esz;
        const dim3 grid((B.nrows + rows - 1) / rows, F);
        const float t = timed([&] {
          k_first<R><<<grid, thr, smem, st>>>(B, rows, ld, only_x ? 1 : 0);
          if (!only_x) k_last<R><<<grid, thr, smem, st>>>(B, rows, ld);
        });
        if (t < tbest) { tbest = t; best = 4 * rows + half; }
      }
    }
    if (status == SWF_OK) ctx->tune.best[xkey] = best;
  }
  if (!only_x) {
    int axes[2], na = 0;
    if (ny > 1) axes[na++] = 1;
    if (nz > 1) axes[na++] = 2;
    const int combos1[1][4] = {{0, 1, 1, 1}};
    const int combos2[3][4] = {{1, 1, 0, 0}, {2, 1, 1, 1}, {1, 0, 0, 1}};
    const int nc = na == 1 ? 1 : 3;
    for (int ci = 0; ci < nc && status == SWF_OK; ++ci) {
      const int* cb = na == 1 ? combos1[ci] : combos2[ci];
      const int axis = na == 1 ? axes[0] : cb[0];
      const int other = axis == 1 ? nz : ny;
      const int n_a = B.g.n[axis];
      const std::string key = tune_key('m', esz, axis * 8 + cb[1] * 4 + cb[2] * 2 + cb[3], n_a, nx, (long)other * F);
      if (ctx->tune.best.count(key)) continue;
      int best = 4 * mid_shape<R>(n_a, nx, (long)other * F).lgtx;
      float tbest = 3.4e38f;
      for (int lg = mid_max_lg<R>(n_a, nx, kPassSmemTune); lg >= 0 && status == SWF_OK; --lg) {
        for (int half = 0; half < 2 && status == SWF_OK; ++half) {
          const MidShape ms = mid_shape_lg<R>(n_a, lg);
          const int ntx = (nx + (1 << lg) - 1) >> lg;
          const dim3 grid(ntx * other, F);
          const float t = timed([&] {
            k_mid<R><<<grid, half ? kThreads / 2 : kThreads, ms.smem, st>>>(B, axis, lg, ms.ld, cb[1], cb[2], cb[3]);
          });
          if (t < tbest) { tbest = t; best = 4 * lg + half; }
        }
      }
      if (status == SWF_OK) ctx->tune.best[key] = best;
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  return status;
}

template <typename R>
static swf_status prepare_args(swf_ctx* ctx, const GridDesc& g, int F, const FieldDesc* fd_host,
                               StageArgs<R>* A, const char* tag, cudaStream_t st) {
  swf_status s = set_smem_attrs<R>();
  if (s != SWF_OK) return s;
  std::memset(A, 0, sizeof(*A));
  A->g = g;
  A->nrows = g.n[1] * g.n[2];
  for (int a = 0; a < 3; ++a) {
    if (!make_march_plan(g.n[a], &A->plan[a])) {
      set_error("grid size must factor into 2, 3 and 5");
      return SWF_EINVAL;
    }
    const void* tw = nullptr;
    s = twiddles(ctx, g.n[a], Prec<R>::is_double, &tw);
    if (s != SWF_OK) return s;
    A->tw[a] = reinterpret_cast<const cpx<R>*>(tw);
  }
  const int nt = g.n[0] + g.n[1] + g.n[2];
  void *pfd = nullptr, *pgr = nullptr, *pgc = nullptr;
  std::string t(tag);
  if ((s = ws_get(ctx, t + ".fd", sizeof(FieldDesc) * F, &pfd)) != SWF_OK) return s;
  if ((s = ws_get(ctx, t + ".greal", sizeof(R) * F * nt, &pgr)) != SWF_OK) return s;
  if ((s = ws_get(ctx, t + ".gcplx", sizeof(cpx<R>) * F * (nt + 4), &pgc)) != SWF_OK) return s;
  void* pkap = nullptr;
  if ((s = ws_get(ctx, t + ".kap", sizeof(R) * nt, &pkap)) != SWF_OK) return s;
  cudaError_t e = cudaMemcpyAsync(pfd, fd_host, sizeof(FieldDesc) * F, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "upload field descriptors");
  A->fd = (const FieldDesc*)pfd;
  A->greal = (const R*)pgr;
  A->gcplx = (const cpx<R>*)pgc;
  A->kap = (const R*)pkap;
  A->inv_n = (R)(1.0 / (double)g.N);
  dim3 tg((nt + 4 + 127) / 128, F);
  {
    ProfScope ps(ctx, "k_tables", st);
    k_tables<R><<<tg, 128, 0, st>>>(A->fd, g, (R*)pgr, (cpx<R>*)pgc);
  }
  ProfScope pk(ctx, "k_kappa_table", st);
  k_kappa_table<R><<<(nt + 127) / 128, 128, 0, st>>>(g, (R*)pkap);
  return SWF_OK;
}

// Runs `pairs` repetitions of two Dormand-Prince steps recorded by `record` (launches only, on
// st), each followed by advancing the march clock by two steps.  Unless kernel timing is on or
// st is the legacy default stream, the pair is captured once into a CUDA graph and replayed:
// one launch per two steps instead of one per kernel.  The slots rotate with period two, so
// the recorded pointers repeat; the stage times come from the device clock.
template <typename Rec>
static swf_status run_step_pairs(swf_ctx* ctx, cudaStream_t st, int pairs, MarchClock* clk, Rec&& record) {
  if (pairs <= 0) return SWF_OK;
  swf_status s = SWF_OK;
  bool graph = !ctx->prof.on && st != 0 && ctx->use_graphs;
  cudaGraphExec_t exec = nullptr;
  long long per_pair = 0;
  if (graph) {
    const long long l0 = ctx->prof.launches;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      graph = false;
    } else {
      s = record();
      k_clock_advance<<<1, 1, 0, st>>>(clk, 2);
      cudaGraph_t gr = nullptr;
      cudaError_t e = cudaStreamEndCapture(st, &gr);
      per_pair = ctx->prof.launches - l0 + 1;
      ctx->prof.launches = l0;
      if (s != SWF_OK) {
        if (gr) cudaGraphDestroy(gr);
        return s;
      }
      if (e != cudaSuccess) return cuda_status(e, "capture of the march steps");
      e = cudaGraphInstantiate(&exec, gr, 0);
      cudaGraphDestroy(gr);
      if (e != cudaSuccess) return cuda_status(e, "instantiate the march graph");
    }
  }
  if (!graph) {
    for (int p = 0; p < pairs && s == SWF_OK; ++p) {
      s = record();
      k_clock_advance<<<1, 1, 0, st>>>(clk, 2);
      ++ctx->prof.launches;
    }
    return s;
  }
  cudaError_t e = cudaSuccess;
  for (int p = 0; p < pairs && e == cudaSuccess; ++p) {
    e = cudaGraphLaunch(exec, st);
    ctx->prof.launches += per_pair;
  }
  // the executable graph is released once its launches have run
  cudaError_t e2 = cudaStreamSynchronize(st);
  cudaGraphExecDestroy(exec);
  if (e != cudaSuccess) return cuda_status(e, "launch the march graph");
  if (e2 != cudaSuccess) return cuda_status(e2, "march graph");
  return SWF_OK;
}

// complex64 fixed-step marches carry the state in float-float: a zeroed low part beside y.
template <typename R>
static swf_status state_low_part(swf_ctx* ctx, const std::string& name, size_t bytes, StageArgs<R>* A,
                                 cudaStream_t st) {
  A->ylo = nullptr;
  if (sizeof(R) != 4) return SWF_OK;
  void* p = nullptr;
  swf_status s = ws_get(ctx, name, bytes, &p);
  if (s != SWF_OK) return s;
  const cudaError_t e = cudaMemsetAsync(p, 0, bytes, st);
  if (e != cudaSuccess) return cuda_status(e, "memset state low part");
  A->ylo = (cpx<R>*)p;
  return SWF_OK;
}

template <typename R>
static swf_status march_impl(swf_ctx* ctx, const GridDesc& g, double t_in, double t_out, int n_steps,
                             int F, const FieldDesc* fd_host, void* psi_out, cudaStream_t st) {
  StageArgs<R> A;
  swf_status s = prepare_args<R>(ctx, g, F, fd_host, &A, "march", st);
  if (s != SWF_OK) return s;
  const size_t state = (size_t)F * 4 * g.N * sizeof(cpx<R>);
  void *py = nullptr, *pT = nullptr, *pk[7];
  if ((s = ws_get(ctx, "march.y", state, &py)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "march.T", state, &pT)) != SWF_OK) return s;
  for (int i = 0; i < 7; ++i) {
    char nm[32];
    std::snprintf(nm, sizeof nm, "march.k%d", i);
    if ((s = ws_get(ctx, nm, state, &pk[i])) != SWF_OK) return s;
  }
  cudaError_t e = cudaMemsetAsync(py, 0, state, st);
  if (e != cudaSuccess) return cuda_status(e, "memset state");
  A.y = (cpx<R>*)py;
  A.T = (cpx<R>*)pT;
  if ((s = state_low_part<R>(ctx, "march.ylo", state, &A, st)) != SWF_OK) return s;
  {
    // shapes by timing, on the slots before they hold anything (the heaviest stage: six inputs)
    StageArgs<R> B = A;
    B.nterm = 6;
    for (int q = 0; q < 6; ++q) {
      B.kin[q] = (const cpx<R>*)pk[q + 1];
      B.coef[q] = 0.0;
    }
    B.write_y = 0;
    B.ystage = nullptr;
    B.kout = (cpx<R>*)pk[0];
    B.t = t_out;
    if ((s = autotune_eval<R>(ctx, B, F, st)) != SWF_OK) return s;
  }
  int slot[7] = {0, 1, 2, 3, 4, 5, 6};
  const double h = (t_in - t_out) / n_steps;
  void* pclk = nullptr;
  if ((s = ws_get(ctx, "march.clock", sizeof(MarchClock), &pclk)) != SWF_OK) return s;
  MarchClock* clk = (MarchClock*)pclk;
  k_clock_set<<<1, 1, 0, st>>>(clk, t_out, h);
  A.clk = clk;
  // Evaluations chain: each one's inverse x pass runs in one launch with the next one's forward x
  // pass (k_last_first), except on grids with x as the only non-trivial axis (one pass per
  // evaluation).  The open evaluation after every second step writes slot 0, as the first
  // evaluation does, so a recorded pair of steps replays unchanged.
  const bool chain = !(g.n[1] == 1 && g.n[2] == 1);
  StageArgs<R> open = A;
  // k_1 = f(t_out, 0)
  A.nterm = 0;
  A.write_y = 0;
  A.kout = (cpx<R>*)pk[slot[0]];
  A.ls = 0;
  A.c = 0.0;
  if ((s = chain ? launch_eval_open<R>(ctx, A, F, st) : launch_eval<R>(ctx, A, F, st)) != SWF_OK) return s;
  open = A;
  // one step at clock offset ls (stage times from the clock: the same arithmetic as
  // tn = t_out + n h, t = tn + c_i h)
  auto step = [&](int ls) -> swf_status {
    for (int i = 1; i < 7; ++i) {
      int nt = 0;
      for (int j = 0; j < i; ++j) {
        if (DP_A[i][j] == 0.0) continue;
        A.kin[nt] = (const cpx<R>*)pk[slot[j]];
        A.coef[nt] = h * DP_A[i][j];
        ++nt;
      }
      A.nterm = nt;
      A.write_y = (i == 6);
      A.kout = (cpx<R>*)pk[slot[i]];
      A.ls = ls;
      A.c = DP_C[i];
      swf_status r = chain ? launch_eval_chain<R>(ctx, open, A, F, st) : launch_eval<R>(ctx, A, F, st);
      if (r != SWF_OK) return r;
      open = A;
    }
    std::swap(slot[0], slot[6]);
    return SWF_OK;
  };
  s = run_step_pairs(ctx, st, n_steps / 2, clk, [&]() -> swf_status {
    swf_status r = step(0);
    return r == SWF_OK ? step(1) : r;
  });
  if (s != SWF_OK) return s;
  if (n_steps % 2 && (s = step(0)) != SWF_OK) return s;
  if (chain && (s = launch_eval_close<R>(ctx, open, F, st)) != SWF_OK) return s;
  e = cudaMemcpyAsync(psi_out, py, state, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "copy psi(t_in)");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "march kernels");
  return SWF_OK;
}

// ---------------------------------------------------------------- step-size control
// Fifth- minus fourth-order weights b_i - b*_i of the Dormand-Prince pair (1980).
static const double DP_DB[7] = {35.0 / 384 - 5179.0 / 57600, 0.0, 500.0 / 1113 - 7571.0 / 16695,
                                125.0 / 192 - 393.0 / 640, -2187.0 / 6784 + 92097.0 / 339200,
                                11.0 / 84 - 187.0 / 2100, -1.0 / 40};

struct ErrWeights {
  double db[7];
};

// part[f][b] = sum over block b's entries of field f of (|e| / (atol + rtol max(|y|, |y_new|)))^2,
// e = h sum_i (b_i - b*_i) k_i, in FP64 (fixed order inside the block).
template <typename R>
__global__ void __launch_bounds__(256) k_step_error(const cpx<R>* __restrict__ y, const cpx<R>* __restrict__ ynew,
                                                    const cpx<R>* k0, const cpx<R>* k1, const cpx<R>* k2,
                                                    const cpx<R>* k3, const cpx<R>* k4, const cpx<R>* k5,
                                                    const cpx<R>* k6, ErrWeights W, const StepControl* ctl,
                                                    size_t per_field, double* part) {
  __shared__ double red[8];
  if (ctl->done) return;
  const int f = blockIdx.y;
  const double h = ctl->h, rtol = ctl->rtol, atol = ctl->atol;
  const cpx<R>* ks[7] = {k0, k1, k2, k3, k4, k5, k6};
  double acc = 0.0;
  const size_t off = (size_t)f * per_field;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < per_field; i += (size_t)gridDim.x * blockDim.x) {
    double ex = 0.0, ey = 0.0;
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      if (W.db[j] == 0.0) continue;
      const cpx<R> kv = ks[j][off + i];
      ex += W.db[j] * (double)kv.x;
      ey += W.db[j] * (double)kv.y;
    }
    const cpx<R> a = y[off + i], b = ynew[off + i];
    const double ya = sqrt((double)a.x * a.x + (double)a.y * a.y), yb = sqrt((double)b.x * b.x + (double)b.y * b.y);
    const double sc = atol + rtol * fmax(ya, yb);
    acc += h * h * (ex * ex + ey * ey) / (sc * sc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < 8; ++w) sum += red[w];
    part[(size_t)f * gridDim.x + blockIdx.x] = sum;
  }
}

// One thread: err = max over fields of the RMS scaled error; accept when err <= 1 (and finite);
// next step h min(10, max(0.2, 0.9 err^(-1/5))), clamped so as not to pass t_in.
__global__ void k_step_control(StepControl* ctl, const double* part, int nb, int F, double count) {
  if (threadIdx.x != 0 || ctl->done) {
    if (threadIdx.x == 0) ctl->ok = 0;
    return;
  }
  double err = 0.0;
  for (int f = 0; f < F; ++f) {
    double sum = 0.0;
    for (int b = 0; b < nb; ++b) sum += part[(size_t)f * nb + b];
    err = fmax(err, sqrt(sum / count));
  }
  if (!(err == err) || isinf(err)) {  // non-finite: stop
    ctl->ok = 0;
    ctl->failed = 1;
    ctl->done = 1;
    return;
  }
  const double fac = err == 0.0 ? 10.0 : fmin(10.0, fmax(0.2, 0.9 * pow(err, -0.2)));
  if (err <= 1.0) {
    ctl->t += ctl->h;
    ctl->ok = 1;
    ctl->accepted += 1;
  } else {
    ctl->ok = 0;
    ctl->rejected += 1;
  }
  double h = ctl->h * fac;
  const double rest = ctl->t_in - ctl->t;
  if (fabs(rest) <= 1e-12 * ctl->span) {
    ctl->done = 1;
  } else if (fabs(h) > fabs(rest)) {
    h = rest;
  }
  ctl->h = h;
  if (!ctl->done && ctl->accepted + ctl->rejected >= ctl->max_attempts) {
    ctl->failed = 1;
    ctl->done = 1;
  }
}

// After an accepted attempt: y <- y_new and k_1 <- k_7 (first same as last).
template <typename R>
__global__ void k_step_accept(const StepControl* ctl, cpx<R>* y, const cpx<R>* ynew, cpx<R>* k1, const cpx<R>* k7,
                              size_t n) {
  if (!ctl->ok) return;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    y[i] = ynew[i];
    k1[i] = k7[i];
  }
}

// Step-size-controlled march (Sec. II.A: Dopri5 with relative and absolute tolerances), from
// t_out with first step h0 toward t_in.  Every attempt (six evaluations, the error norm, the
// controller, the copy-in of an accepted step) is one CUDA graph replay; nothing is decided on
// the host: after t_in (or a failure) the remaining replays of a chunk do nothing.  The host
// reads the controller's state once per chunk of replays.
// Runs step attempts recorded by `attempt` (launches only, on st) until the controller in ctl
// reports t_in reached or a failure: chunks of 8, 16, .. 64 attempts as CUDA-graph replays
// (kernel by kernel when timing is on), the controller's state read once per chunk into *out.
// Condition of the device-side attempt loop: another attempt while the controller is not done
// (the controller itself stops at max_attempts; the bound is repeated here so that the loop ends
// whatever the state).
__global__ void k_attempt_condition(cudaGraphConditionalHandle h, const StepControl* ctl) {
  const bool more = !ctl->done && ctl->accepted + ctl->rejected < ctl->max_attempts;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

// The whole controlled march as one graph launch: a while node whose body is one attempt and
// k_attempt_condition, so that accepting, rejecting and stopping are decided on the device and
// the host reads the controller's state once, at the end.  *built = false (nothing launched) when
// the graph cannot be built here; the caller then runs its host loop.
template <typename Att>
static swf_status attempts_on_device(swf_ctx* ctx, cudaStream_t st, const StepControl* ctl, Att&& attempt,
                                     StepControl* out, bool* built) {
  *built = false;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) {
    cudaGetLastError();
    return SWF_OK;
  }
  swf_status s = SWF_OK;
  long long per_attempt = 0;
  cudaGraphConditionalHandle h;
  // the parameter union has no default constructor: zeroed storage
  alignas(cudaGraphNodeParams) unsigned char np_raw[sizeof(cudaGraphNodeParams)];
  std::memset(np_raw, 0, sizeof(np_raw));
  cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(np_raw);
  cudaGraphNode_t node;
  bool ok = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
  if (ok) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
  }
  if (ok) ok = cudaStreamBeginCaptureToGraph(st, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    const long long l0 = ctx->prof.launches;
    s = attempt();
    k_attempt_condition<<<1, 1, 0, st>>>(h, ctl);
    cudaGraph_t body = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(st, &body);
    per_attempt = ctx->prof.launches - l0 + 1;
    ctx->prof.launches = l0;
    ok = s == SWF_OK && ec == cudaSuccess && cudaGraphInstantiate(&exec, g, 0) == cudaSuccess;
  }
  cudaGraphDestroy(g);
  if (s != SWF_OK) {
    if (exec) cudaGraphExecDestroy(exec);
    return s;
  }
  if (!ok) {
    if (exec) cudaGraphExecDestroy(exec);
    cudaGetLastError();  // an unsupported graph form is not an error of the march
    return SWF_OK;
  }
  *built = true;
  cudaError_t e = cudaGraphLaunch(exec, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, ctl, sizeof(StepControl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaGraphExecDestroy(exec);
  if (e != cudaSuccess) return cuda_status(e, "step-size-controlled march (device loop)");
  ctx->prof.launches += per_attempt * (out->accepted + out->rejected);
  ctx->device_loop_marches += 1;
  return SWF_OK;
}

template <typename Att>
static swf_status run_attempts(swf_ctx* ctx, cudaStream_t st, int max_attempts, const StepControl* ctl,
                               Att&& attempt, StepControl* out) {
  swf_status s = SWF_OK;
  cudaError_t e = cudaSuccess;
  bool graph = !ctx->prof.on && st != 0 && ctx->use_graphs;
  cudaGraphExec_t exec = nullptr;
  long long per_attempt = 0;
  if (graph) {
    bool built = false;
    s = attempts_on_device(ctx, st, ctl, attempt, out, &built);
    if (s != SWF_OK || built) return s;
  }
  if (graph) {
    const long long l0 = ctx->prof.launches;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      graph = false;
    } else {
      s = attempt();
      cudaGraph_t gr = nullptr;
      e = cudaStreamEndCapture(st, &gr);
      per_attempt = ctx->prof.launches - l0;
      ctx->prof.launches = l0;
      if (s != SWF_OK) {
        if (gr) cudaGraphDestroy(gr);
        return s;
      }
      if (e != cudaSuccess) return cuda_status(e, "capture of the step attempt");
      e = cudaGraphInstantiate(&exec, gr, 0);
      cudaGraphDestroy(gr);
      if (e != cudaSuccess) return cuda_status(e, "instantiate the step attempt");
    }
  }
  StepControl hc{};
  int chunk = 8, attempts = 0;
  while (true) {
    for (int a = 0; a < chunk; ++a) {
      if (graph) {
        e = cudaGraphLaunch(exec, st);
        ctx->prof.launches += per_attempt;
        if (e != cudaSuccess) break;
      } else if ((s = attempt()) != SWF_OK) {
        if (exec) cudaGraphExecDestroy(exec);
        return s;
      }
    }
    attempts += chunk;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, ctl, sizeof(StepControl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess || hc.done) break;
    if (attempts > max_attempts + chunk) {  // the controller stops at max_attempts; this is a backstop
      hc.failed = 1;
      break;
    }
    chunk = std::min(chunk * 2, 64);
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (e != cudaSuccess) return cuda_status(e, "step-size-controlled march");
  *out = hc;
  return SWF_OK;
}

template <typename R>
static swf_status march_adaptive_impl(swf_ctx* ctx, const GridDesc& g, double t_in, double t_out, double h0,
                                      int max_attempts, int F, const FieldDesc* fd_host, void* psi_out,
                                      cudaStream_t st) {
  StageArgs<R> A;
  swf_status s = prepare_args<R>(ctx, g, F, fd_host, &A, "march", st);
  if (s != SWF_OK) return s;
  const size_t per_field = (size_t)4 * g.N;
  const size_t state = (size_t)F * per_field * sizeof(cpx<R>);
  void *py = nullptr, *pyn = nullptr, *pT = nullptr, *pk[7], *pctl = nullptr, *ppart = nullptr;
  if ((s = ws_get(ctx, "march.y", state, &py)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "march.ynew", state, &pyn)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "march.T", state, &pT)) != SWF_OK) return s;
  for (int i = 0; i < 7; ++i) {
    char nm[32];
    std::snprintf(nm, sizeof nm, "march.k%d", i);
    if ((s = ws_get(ctx, nm, state, &pk[i])) != SWF_OK) return s;
  }
  const int nbe = (int)std::max<size_t>(1, std::min<size_t>((per_field + 4095) / 4096, 64));
  if ((s = ws_get(ctx, "march.ctl", sizeof(StepControl), &pctl)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "march.err_part", sizeof(double) * (size_t)nbe * F, &ppart)) != SWF_OK) return s;
  cudaError_t e = cudaMemsetAsync(py, 0, state, st);
  if (e != cudaSuccess) return cuda_status(e, "memset state");
  StepControl c0{};
  c0.t = t_out;
  c0.h = (t_in < t_out) ? -std::fabs(h0) : std::fabs(h0);
  if (std::fabs(c0.h) > std::fabs(t_in - t_out)) c0.h = t_in - t_out;
  c0.t_in = t_in;
  c0.span = std::fabs(t_in - t_out);
  c0.rtol = ctx->rtol;
  c0.atol = ctx->atol;
  c0.max_attempts = max_attempts;
  StepControl* ctl = (StepControl*)pctl;
  e = cudaMemcpyAsync(ctl, &c0, sizeof(StepControl), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "upload step control");
  A.y = (cpx<R>*)py;
  A.T = (cpx<R>*)pT;
  {
    StageArgs<R> B = A;  // shapes by timing, before the slots hold anything
    B.nterm = 6;
    for (int q = 0; q < 6; ++q) {
      B.kin[q] = (const cpx<R>*)pk[q + 1];
      B.coef[q] = 0.0;
    }
    B.write_y = 0;
    B.ystage = nullptr;
    B.kout = (cpx<R>*)pk[0];
    B.t = t_out;
    if ((s = autotune_eval<R>(ctx, B, F, st)) != SWF_OK) return s;
  }
  // k_1 = f(t_out, 0)
  A.nterm = 0;
  A.write_y = 0;
  A.kout = (cpx<R>*)pk[0];
  A.t = t_out;
  if ((s = launch_eval<R>(ctx, A, F, st)) != SWF_OK) return s;
  A.ctl = ctl;
  A.ynew = (cpx<R>*)pyn;
  ErrWeights W;
  for (int j = 0; j < 7; ++j) W.db[j] = DP_DB[j];
  // the evaluations of an attempt chain through k_last_first; the attempt's last one is closed
  // before the error estimate reads k_7
  const bool chain = !(g.n[1] == 1 && g.n[2] == 1);
  auto attempt = [&]() -> swf_status {
    StageArgs<R> open = A;
    for (int i = 1; i < 7; ++i) {
      int nt = 0;
      for (int j = 0; j < i; ++j) {
        if (DP_A[i][j] == 0.0) continue;
        A.kin[nt] = (const cpx<R>*)pk[j];
        A.coef[nt] = DP_A[i][j];  // times the device-held h in k_first
        ++nt;
      }
      A.nterm = nt;
      A.write_y = (i == 6);
      A.kout = (cpx<R>*)pk[i];
      A.c = DP_C[i];
      swf_status r = !chain ? launch_eval<R>(ctx, A, F, st)
                            : (i == 1 ? launch_eval_open<R>(ctx, A, F, st) : launch_eval_chain<R>(ctx, open, A, F, st));
      if (r != SWF_OK) return r;
      open = A;
    }
    if (chain) {
      swf_status r = launch_eval_close<R>(ctx, open, F, st);
      if (r != SWF_OK) return r;
    }
    {
      ProfScope ps(ctx, "k_step_error", st);
      k_step_error<R><<<dim3(nbe, F), 256, 0, st>>>(
          (const cpx<R>*)py, (const cpx<R>*)pyn, (const cpx<R>*)pk[0], (const cpx<R>*)pk[1], (const cpx<R>*)pk[2],
          (const cpx<R>*)pk[3], (const cpx<R>*)pk[4], (const cpx<R>*)pk[5], (const cpx<R>*)pk[6], W, ctl, per_field,
          (double*)ppart);
    }
    {
      ProfScope ps(ctx, "k_step_control", st);
      k_step_control<<<1, 32, 0, st>>>(ctl, (const double*)ppart, nbe, F, (double)per_field);
    }
    {
      ProfScope ps(ctx, "k_step_accept", st);
      const size_t n = (size_t)F * per_field;
      k_step_accept<R><<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(
          ctl, (cpx<R>*)py, (const cpx<R>*)pyn, (cpx<R>*)pk[0], (const cpx<R>*)pk[6], n);
    }
    return SWF_OK;
  };
  StepControl hc{};
  if ((s = run_attempts(ctx, st, max_attempts, ctl, attempt, &hc)) != SWF_OK) return s;
  ctx->last_accepted = hc.accepted;
  ctx->last_rejected = hc.rejected;
  if (hc.failed) {
    set_error("step-size-controlled march: no convergence (too many attempts or a non-finite error)");
    return SWF_ENUMERIC;
  }
  e = cudaMemcpyAsync(psi_out, py, state, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "copy psi(t_in)");
  return SWF_OK;
}

swf_status march_adaptive(swf_ctx* ctx, const GridDesc& g, double t_in, double t_out, double h0, int max_attempts,
                          int n_f, const FieldDesc* fd_host, swf_precision prec, void* psi_out, cudaStream_t st) {
  if (prec == SWF_C64)
    return march_adaptive_impl<float>(ctx, g, t_in, t_out, h0, max_attempts, n_f, fd_host, psi_out, st);
  return march_adaptive_impl<double>(ctx, g, t_in, t_out, h0, max_attempts, n_f, fd_host, psi_out, st);
}

// psi_out[f] = psi_u[rep[f]] with the components {1, 2} times sgn[f] (+1 or -1).
template <typename R>
__global__ void k_expand_fields(const cpx<R>* __restrict__ psi_u, const int* __restrict__ rep,
                                const int* __restrict__ sgn, size_t N, cpx<R>* __restrict__ psi_out) {
  const int f = blockIdx.y;
  const int c = blockIdx.z;
  const R s = (c == 1 || c == 2) ? (R)sgn[f] : (R)1;
  const cpx<R>* src = psi_u + ((size_t)rep[f] * 4 + c) * N;
  cpx<R>* dst = psi_out + ((size_t)f * 4 + c) * N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = s * src[i];
}

static bool same_desc_but_spinor(const FieldDesc& a, const FieldDesc& b) {
  if (a.kind != b.kind || a.acomp != b.acomp || a.e0 != b.e0 || a.tsign != b.tsign) return false;
  for (int k = 0; k < 8; ++k)
    if (a.prm[k] != b.prm[k]) return false;
  for (int k = 0; k < 3; ++k)
    if (a.K[k] != b.K[k] || a.pmom[k] != b.pmom[k]) return false;
  return true;
}

// Fields whose march repeats another's: the same field, background momentum and energy, and a
// background spinor that is the same or (when the spin along z is conserved) the same with the
// components {1, 2} negated.  The second case is the other spin: R_- = diag(1, -1, -1, 1) R_+,
// and (1 +- p-slash), alpha^x, alpha^y, beta and A_0 never mix {0, 3} with {1, 2} when p_z = 0,
// the z axis is trivial and A_3 = 0, so the scattered wave of the other spin is the same wave
// with {1, 2} negated, exactly.  rep[f] indexes the unique list; sgn[f] is the sign of {1, 2}.
static int dedupe_fields(const GridDesc& g, int n_f, const FieldDesc* fd, std::vector<int>& rep,
                         std::vector<int>& sgn, std::vector<FieldDesc>& uniq) {
  rep.assign(n_f, 0);
  sgn.assign(n_f, 1);
  uniq.clear();
  std::vector<int> first;  // field index of each unique entry
  for (int f = 0; f < n_f; ++f) {
    const FieldDesc& a = fd[f];
    const bool zsym = g.n[2] == 1 && a.K[2] == 0.0 && a.acomp != 3;
    int found = -1, sign = 1;
    for (size_t u = 0; u < uniq.size() && found < 0; ++u) {
      const FieldDesc& b = uniq[u];
      if (!same_desc_but_spinor(a, b)) continue;
      bool eq = true, flip = zsym;
      for (int k = 0; k < 8; ++k) {
        const bool in_b = (k >> 1) == 1 || (k >> 1) == 2;  // components 1 and 2
        if (a.w[k] != b.w[k]) eq = false;
        if (a.w[k] != (in_b ? -b.w[k] : b.w[k])) flip = false;
      }
      if (eq) { found = (int)u; sign = 1; }
      else if (flip) { found = (int)u; sign = -1; }
    }
    if (found < 0) {
      found = (int)uniq.size();
      uniq.push_back(a);
      first.push_back(f);
    }
    rep[f] = found;
    sgn[f] = sign;
  }
  return (int)uniq.size();
}

// Sizes the pass-kernel march's workspace for F fields (the buffers prepare_args and march_impl
// take) without touching the device: growing a workspace buffer frees the old one, which waits
// for the whole device, so march_split does it before the fused kernel starts.
template <typename R>
static swf_status reserve_march(swf_ctx* ctx, const GridDesc& g, int F) {
  const int nt = g.n[0] + g.n[1] + g.n[2];
  const size_t state = (size_t)F * 4 * g.N * sizeof(cpx<R>);
  void* p = nullptr;
  swf_status s;
  if ((s = ws_get(ctx, "march.fd", sizeof(FieldDesc) * F, &p)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "march.greal", sizeof(R) * F * nt, &p)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "march.gcplx", sizeof(cpx<R>) * F * (nt + 4), &p)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "march.y", state, &p)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "march.T", state, &p)) != SWF_OK) return s;
  if (sizeof(R) == 4 && (s = ws_get(ctx, "march.ylo", state, &p)) != SWF_OK) return s;
  for (int i = 0; i < 7; ++i) {
    char nm[32];
    std::snprintf(nm, sizeof nm, "march.k%d", i);
    if ((s = ws_get(ctx, nm, state, &p)) != SWF_OK) return s;
  }
  if ((s = ws_get(ctx, "march.clock", sizeof(MarchClock), &p)) != SWF_OK) return s;
  for (int a = 0; a < 3; ++a) {
    const void* tw = nullptr;
    if ((s = twiddles(ctx, g.n[a], Prec<R>::is_double, &tw)) != SWF_OK) return s;
  }
  return SWF_OK;
}

// The fused kernel's 16-CTA clusters (one CTA per SM) fit once per GPC, so some SMs stay idle
// (on GB300: 7 clusters on 112 of 152 SMs).  Moving some fields to the pass kernels, run
// concurrently on those SMs, shortens the march when they finish within the fused kernel's
// time.  With R = ceil(2 n_f / ncl) rounds of sectors per cluster, removing r rounds leaves
// n_1 = floor((R - r) ncl / 2) fields to the clusters and n_2 = n_f - n_1 to the pass kernels,
// which take about alpha n_2 rounds' time on the free SMs.  alpha was measured with 40 free SMs
// on (2+1)D 256^2 complex64 marches: with the pushed-transpose kernel and the chained x passes,
// 16 fields took 2.75 s on the free SMs while the fused launch took 32 rounds in 2.78 s
// (alpha = 2.0); rounds of the pulled-transpose kernel are 1.46 times longer (alpha = 1.37).
// alpha scales with 40 / (free SMs).  The largest r with alpha n_2 <= R - r is taken.
int fused_split_count(int n_f, int ncl, int n_sm, int variant) {
  const int free_sm = n_sm - kFusedClusterCtas * ncl;
  if (ncl < 1 || free_sm < 16 || n_f < 16) return 0;
  const double alpha = (variant == 3 ? 2.0 : 1.37) * 40.0 / free_sm;
  const int R = (2 * n_f + ncl - 1) / ncl;
  int best = 0;
  for (int r = 1; r < R; ++r) {
    const int n1 = ((R - r) * ncl) / 2;
    const int n2 = n_f - n1;
    if (n2 <= 0) continue;
    if (alpha * n2 > (double)(R - r)) break;
    best = n2;
  }
  return best;
}

// The fused kernel on the first n_f - n2 fields (stream st) and, concurrently, the pass kernels
// on the last n2 fields (the context's auxiliary stream), which take the SMs that the fused
// kernel's clusters leave free.  The auxiliary stream starts after the work already queued on
// st and st continues after both.  complex64 only (the fused kernel's precision).
static swf_status march_split(swf_ctx* ctx, const GridDesc& g, double t_in, double t_out, int n_steps, int n_f,
                              int n2, const FieldDesc* fd_host, void* psi_out, cudaStream_t st) {
  cudaError_t e;
  if (!ctx->aux) {
    if ((e = cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking)) != cudaSuccess)
      return cuda_status(e, "auxiliary stream");
    for (int i = 0; i < 2; ++i)
      if ((e = cudaEventCreateWithFlags(&ctx->aux_ev[i], cudaEventDisableTiming)) != cudaSuccess)
        return cuda_status(e, "auxiliary stream events");
  }
  const int n1 = n_f - n2;
  swf_status s = reserve_march<float>(ctx, g, n2);
  if (s != SWF_OK) return s;
  if ((e = cudaEventRecord(ctx->aux_ev[0], st)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(ctx->aux, ctx->aux_ev[0], 0)) != cudaSuccess)
    return cuda_status(e, "order the auxiliary stream");
  s = march_fused(ctx, g, t_in, t_out, n_steps, n1, fd_host, psi_out, st);
  if (s != SWF_OK) return s;
  cpx<float>* out2 = (cpx<float>*)psi_out + (size_t)n1 * 4 * g.N;
  s = march_impl<float>(ctx, g, t_in, t_out, n_steps, n2, fd_host + n1, out2, ctx->aux);
  if (s != SWF_OK) return s;
  if ((e = cudaEventRecord(ctx->aux_ev[1], ctx->aux)) != cudaSuccess ||
      (e = cudaStreamWaitEvent(st, ctx->aux_ev[1], 0)) != cudaSuccess)
    return cuda_status(e, "join the auxiliary stream");
  return SWF_OK;
}

static swf_status march_unique(swf_ctx* ctx, const GridDesc& g, double t_in, double t_out, int n_steps, int n_f,
                               const FieldDesc* fd_host, swf_precision prec, void* psi_out, cudaStream_t st,
                               int adaptive) {
  if (adaptive)  // first step (t_in - t_out)/n_steps, at most 100 n_steps + 100 attempts
    return march_adaptive(ctx, g, t_in, t_out, (t_in - t_out) / n_steps, 100 * n_steps + 100, n_f, fd_host, prec,
                          psi_out, st);
  if (ctx->use_fused && fused_applicable(g, n_f, fd_host, prec)) {
    const int n2 = (ctx->sm_split && ctx->fused_variant != 2)
                       ? fused_split_count(n_f, fused_resident_clusters(ctx), sm_count(), ctx->fused_variant)
                       : 0;
    if (n2 > 0) return march_split(ctx, g, t_in, t_out, n_steps, n_f, n2, fd_host, psi_out, st);
    swf_status s = march_fused(ctx, g, t_in, t_out, n_steps, n_f, fd_host, psi_out, st);
    if (s != SWF_EUNSUPPORTED) return s;
    ctx->use_fused = false;  // the cluster shape cannot be resident here: pass kernels from now on
  }
  if (prec == SWF_C64) return march_impl<float>(ctx, g, t_in, t_out, n_steps, n_f, fd_host, psi_out, st);
  return march_impl<double>(ctx, g, t_in, t_out, n_steps, n_f, fd_host, psi_out, st);
}

swf_status march_fields(swf_ctx* ctx, const GridDesc& g, double t_in, double t_out, int n_steps,
                        int n_f, const FieldDesc* fd_host, swf_precision prec, void* psi_out,
                        cudaStream_t st, int adaptive) {
  std::vector<int> rep, sgn;
  std::vector<FieldDesc> uniq;
  const int n_u = ctx->dedupe ? dedupe_fields(g, n_f, fd_host, rep, sgn, uniq) : n_f;
  ctx->fields_marched += n_u;
  if (n_u == n_f) return march_unique(ctx, g, t_in, t_out, n_steps, n_f, fd_host, prec, psi_out, st, adaptive);
  const size_t elem = prec == SWF_C64 ? 8 : 16;
  void *pu = nullptr, *ptab = nullptr;
  swf_status s = ws_get(ctx, "march.unique", (size_t)n_u * 4 * g.N * elem, &pu);
  if (s != SWF_OK) return s;
  if ((s = ws_get(ctx, "march.unique_map", sizeof(int) * 2 * (size_t)n_f, &ptab)) != SWF_OK) return s;
  if ((s = march_unique(ctx, g, t_in, t_out, n_steps, n_u, uniq.data(), prec, pu, st, adaptive)) != SWF_OK) return s;
  std::vector<int> tab(rep);
  tab.insert(tab.end(), sgn.begin(), sgn.end());
  cudaError_t e = cudaMemcpyAsync(ptab, tab.data(), sizeof(int) * 2 * (size_t)n_f, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "upload field map");
  const dim3 grid((unsigned)std::min<size_t>((g.N + 255) / 256, 1024), n_f, 4);
  ProfScope ps(ctx, "k_expand_fields", st);
  if (prec == SWF_C64)
    k_expand_fields<float><<<grid, 256, 0, st>>>((const cpx<float>*)pu, (const int*)ptab, (const int*)ptab + n_f,
                                                 (size_t)g.N, (cpx<float>*)psi_out);
  else
    k_expand_fields<double><<<grid, 256, 0, st>>>((const cpx<double>*)pu, (const int*)ptab, (const int*)ptab + n_f,
                                                  (size_t)g.N, (cpx<double>*)psi_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "expand fields");
  // the host table must outlive its asynchronous upload
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "expand fields");
  return SWF_OK;
}

template <typename R>
static swf_status rhs_impl(swf_ctx* ctx, const GridDesc& g, const FieldDesc& fd, double t,
                           const void* psi, void* out, cudaStream_t st) {
  StageArgs<R> A;
  swf_status s = prepare_args<R>(ctx, g, 1, &fd, &A, "rhs", st);
  if (s != SWF_OK) return s;
  void* pT = nullptr;
  if ((s = ws_get(ctx, "rhs.T", (size_t)4 * g.N * sizeof(cpx<R>), &pT)) != SWF_OK) return s;
  A.y = const_cast<cpx<R>*>((const cpx<R>*)psi);  // read only: write_y = 0
  A.T = (cpx<R>*)pT;
  A.kout = (cpx<R>*)out;
  A.nterm = 0;
  A.write_y = 0;
  A.t = t;
  if ((s = launch_eval<R>(ctx, A, 1, st)) != SWF_OK) return s;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "rhs kernels");
  return SWF_OK;
}

swf_status rhs_eval(swf_ctx* ctx, const GridDesc& g, const FieldDesc& fd, swf_precision prec,
                    double t, const void* psi, void* out, cudaStream_t st) {
  if (prec == SWF_C64) return rhs_impl<float>(ctx, g, fd, t, psi, out, st);
  return rhs_impl<double>(ctx, g, fd, t, psi, out, st);
}

}  // namespace swf

// ---------------------------------------------------------------- right-hand side in caller scratch
namespace swf {

template <typename R>
__global__ void k_twiddles_into(cpx<R>* tw, int n) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(-2.0 * m / (double)n, &s, &c);
    tw[m] = mk<R>((R)c, (R)s);
  }
}

static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Stores a field descriptor passed by value (kernel parameters are copied at launch, so no host
// memory is referenced once the launch returns).
__global__ void k_store_field_desc(FieldDesc fd, FieldDesc* dst) { *dst = fd; }

size_t rhs_scratch_bytes(const GridDesc& g, swf_precision prec) {
  const size_t e = prec == SWF_C64 ? 8 : 16, r = prec == SWF_C64 ? 4 : 8;
  const size_t nt = g.n[0] + g.n[1] + g.n[2];
  return align256(4 * (size_t)g.N * e) + align256(sizeof(FieldDesc)) + 2 * align256(nt * r) +
         align256((nt + 4) * e) + 3 * align256(512 * e);
}

// Same evaluation as rhs_eval, with every buffer (FFT workspace, field tables, twiddles, the
// field descriptor) carved out of `scratch` instead of the context's workspace; no device
// memory is allocated.
template <typename R>
static swf_status rhs_scratch_impl(const GridDesc& g, const FieldDesc& fd, double t, const void* psi, void* out,
                                   unsigned char* scratch, cudaStream_t st) {
  swf_status s = set_smem_attrs<R>();
  if (s != SWF_OK) return s;
  const int nt = g.n[0] + g.n[1] + g.n[2];
  unsigned char* p = scratch;
  cpx<R>* T = (cpx<R>*)p;
  p += align256((size_t)4 * g.N * sizeof(cpx<R>));
  FieldDesc* dfd = (FieldDesc*)p;
  p += align256(sizeof(FieldDesc));
  R* greal = (R*)p;
  p += align256((size_t)nt * sizeof(R));
  cpx<R>* gcplx = (cpx<R>*)p;
  p += align256((size_t)(nt + 4) * sizeof(cpx<R>));
  R* kap = (R*)p;
  p += align256((size_t)nt * sizeof(R));
  StageArgs<R> A;
  std::memset(&A, 0, sizeof(A));
  A.g = g;
  A.nrows = g.n[1] * g.n[2];
  for (int a = 0; a < 3; ++a) {
    if (!make_march_plan(g.n[a], &A.plan[a])) {
      set_error("grid size must factor into 2, 3 and 5");
      return SWF_EINVAL;
    }
    cpx<R>* tw = (cpx<R>*)p;
    p += align256(512 * sizeof(cpx<R>));
    k_twiddles_into<R><<<(g.n[a] + 127) / 128, 128, 0, st>>>(tw, g.n[a]);
    A.tw[a] = tw;
  }
  k_store_field_desc<<<1, 1, 0, st>>>(fd, dfd);
  k_tables<R><<<dim3((nt + 4 + 127) / 128, 1), 128, 0, st>>>(dfd, g, greal, gcplx);
  k_kappa_table<R><<<(nt + 127) / 128, 128, 0, st>>>(g, kap);
  A.kap = kap;
  A.inv_n = (R)(1.0 / (double)g.N);
  A.fd = dfd;
  A.greal = greal;
  A.gcplx = gcplx;
  A.y = const_cast<cpx<R>*>((const cpx<R>*)psi);
  A.T = T;
  A.kout = (cpx<R>*)out;
  A.t = t;
  s = launch_eval<R>(nullptr, A, 1, st);
  if (s != SWF_OK) return s;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "rhs kernels");
  return SWF_OK;
}

swf_status rhs_eval_scratch(const GridDesc& g, const FieldDesc& fd, swf_precision prec, double t, const void* psi,
                            void* out, void* scratch, cudaStream_t st) {
  if (prec == SWF_C64) return rhs_scratch_impl<float>(g, fd, t, psi, out, (unsigned char*)scratch, st);
  return rhs_scratch_impl<double>(g, fd, t, psi, out, (unsigned char*)scratch, st);
}

}  // namespace swf

// ---------------------------------------------------------------- Breit-Wheeler march (Sec. IV)
namespace swf {

// Dormand-Prince 5th-order weights b_i (the 7th is zero; FSAL)

// Photon plane-wave factor exp(i k.x) per axis for each instance (trivial axes: 1).
template <typename R>
__global__ void k_photon_tables(const double* photon, GridDesc g, int n_inst, cpx<R>* kph) {
  const int nt = g.n[0] + g.n[1] + g.n[2];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_inst * nt; i += gridDim.x * blockDim.x) {
    const int inst = i / nt;
    int j = i % nt, axis = 0;
    while (j >= g.n[axis]) { j -= g.n[axis]; ++axis; }
    const double xc = g.n[axis] > 1 ? g.x0[axis] + j * g.dx[axis] : 0.0;
    double s, c;
    sincos(photon[6 * inst + axis] * xc, &s, &c);
    kph[i] = mk<R>((R)c, (R)s);
  }
}

// Per instance, step and stage (Dormand-Prince nodes c_i) at t = t_out + (step + c_i) h, with the
// quadrature weight w_i = h b_{i+1} for i = 2..5 and h b_1 (of the next step) for the last stage,
// 0 elsewhere.  form 1: the background time phases of U and V and w_i dx^d e^{-i k0 t} (the
// integrand of Eq. 17 vanishes at the first stage, psi_s(t_out) = 0).  form 2 (Eqs. 30-33):
// w_i e^{-i(q0 - k0)t} and w_i e^{i(p0 - k0)t} for the direct transforms of the U and V waves
// and w_i e^{-i k0 t} for the mode sum; the first stage of the march carries h b_1 (the source
// term is not zero there).  FP64, computed once per march so that the integrand kernels need none.
__global__ void k_bw_phase_table(const FieldDesc* fd, const double* photon, int n_pi, int n_ph, int n_steps,
                                 double t_out, double h, double cell, int form, cpx<double>* tab) {
  const double DPc[7] = {0.0, 0.2, 0.3, 0.8, 8.0 / 9.0, 1.0, 1.0};
  const double DPb[7] = {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0.0};
  const long total = (long)n_pi * n_steps * 7;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const int pi = (int)(e / (7L * n_steps));  // photon-instance; its waves are those of instance pi / n_ph
    const int inst = pi / n_ph;
    const int step = (int)((e / 7) % n_steps), i = (int)(e % 7);
    const double t = t_out + (step + DPc[i]) * h;
    double w = (i >= 2 && i <= 5) ? h * DPb[i] : (i == 6 && step + 1 < n_steps ? h * DPb[0] : 0.0);
    if (form == 2 && i == 0 && step == 0) w = h * DPb[0];
    double sn, cs;
    const FieldDesc& FU = fd[2 * inst];
    const FieldDesc& FV = fd[2 * inst + 1];
    const double k0 = sqrt(photon[6 * pi] * photon[6 * pi] + photon[6 * pi + 1] * photon[6 * pi + 1] +
                           photon[6 * pi + 2] * photon[6 * pi + 2]);
    if (form == 2) {
      sincos(-(FV.e0 - k0) * t, &sn, &cs);
      tab[3 * e] = mk<double>(w * cs, w * sn);
      sincos((FU.e0 - k0) * t, &sn, &cs);
      tab[3 * e + 1] = mk<double>(w * cs, w * sn);
      sincos(-k0 * t, &sn, &cs);
      tab[3 * e + 2] = mk<double>(w * cs, w * sn);
      continue;
    }
    sincos(FU.tsign * FU.e0 * t, &sn, &cs);
    tab[3 * e] = mk<double>(cs, sn);
    sincos(FV.tsign * FV.e0 * t, &sn, &cs);
    tab[3 * e + 1] = mk<double>(cs, sn);
    sincos(-k0 * t, &sn, &cs);
    tab[3 * e + 2] = mk<double>(w * cell * cs, w * cell * sn);
  }
}

// Sum over the 32 lanes of a warp in the march precision (lane 0 holds it); the integrand kernels
// add the warps' sums of a block in FP64.  FP64 is scarce on GB300: a shuffle tree in FP64 per
// block and value cost more than the integrand itself.
template <typename R>
__device__ __forceinline__ cpx<R> warp_sum(cpx<R> v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, off);
    v.y += __shfl_down_sync(0xffffffffu, v.y, off);
  }
  return v;
}

// (alpha . eps) v for a real polarisation eps (Dirac representation), every rounding fixed (the
// integrand must give the same bits in every launch variant).
template <typename R>
__device__ __forceinline__ void alpha_eps(const R* e, const cpx<R>* v, cpx<R>* o) {
  // sigma.eps (u0, u1) = (ez u0 + ex u1 - i ey u1, ex u0 + i ey u0 - ez u1)
  const R mz = -e[2];
  o[0] = xadd(xadd(xscale(e[2], v[2]), xscale(e[0], v[3])), xscale(e[1], mul_mi(v[3])));
  o[1] = xadd(xadd(xscale(e[0], v[2]), xscale(e[1], mul_i(v[2]))), xscale(mz, v[3]));
  o[2] = xadd(xadd(xscale(e[2], v[0]), xscale(e[0], v[1])), xscale(e[1], mul_mi(v[1])));
  o[3] = xadd(xadd(xscale(e[0], v[0]), xscale(e[1], mul_i(v[0]))), xscale(mz, v[1]));
}

// The three integrands of Eq. 17, dx^d sum_x U_a^+ (alpha.eps) V_b exp(-ikx), for (ss, bs, sb)
// at the stage values, integrated with weight w (= h b_i).  Block (b, pi) sums the sites
// j = b*256 + threadIdx.x (stride gridDim.x*256) of photon-instance pi (photon pi % n_ph of
// instance pi / n_ph: several photons share one march) and adds w dx^d e^{-i k0 t}
// (from the phase table) times its sum to its own accumulator acc[pi][b][3] (FP64; no other block touches it, so
// the march's sum is deterministic); k_mdot_final adds the accumulators in a fixed order.
// Block (bx, by) of a launch with nbx blocks per row.
template <typename R, int NPH>
__device__ __forceinline__ void mdot_body(const cpx<R>* __restrict__ ys, const cpx<R>* gcplx, const cpx<R>* kph,
                                          const double* photon, const GridDesc& g,
                                          const cpx<double>* __restrict__ ptab, const MarchClock* clk, int ls,
                                          int stage, int tab_stride, int n_ph, cpx<double>* acc, int bx, int by,
                                          int nbx) {
  const long tab_row = (long)(clk->step + ls) * 7 + stage;
  __shared__ cpx<double> red[8][3 * NPH];
  // block row: instance inst, photons j0 .. j0 + nj - 1 (photon-instances pi0 + jj); U and V are
  // loaded once per site for the NPH photons of the block
  const int nchunk = (n_ph + NPH - 1) / NPH;
  const int inst = by / nchunk;
  const int j0 = (by % nchunk) * NPH;
  const int nj = min(NPH, n_ph - j0);
  const int pi0 = inst * n_ph + j0;
  const int nt = g.n[0] + g.n[1] + g.n[2];
  const cpx<R>* tu = gcplx + (size_t)(2 * inst) * (nt + 4);
  const cpx<R>* tv = gcplx + (size_t)(2 * inst + 1) * (nt + 4);
  // the U and V time phases are the same in every photon's row of the phase table
  const cpx<double>* trow0 = ptab + 3 * (tab_row + (long)pi0 * tab_stride);
  const cpx<R> tfu = cvt<R>(trow0[0]), tfv = cvt<R>(trow0[1]);
  R eps[NPH][3];
  const cpx<R>* kp[NPH];
#pragma unroll
  for (int jj = 0; jj < NPH; ++jj) {
    const int pj = pi0 + min(jj, nj - 1);  // a partial last chunk repeats its last photon (not stored)
    kp[jj] = kph + (size_t)pj * nt;
    for (int a = 0; a < 3; ++a) eps[jj][a] = (R)photon[6 * pj + 3 + a];
  }
  const cpx<R>* U = ys + (size_t)(2 * inst) * 4 * g.N;
  const cpx<R>* V = ys + (size_t)(2 * inst + 1) * 4 * g.N;
  // per-thread sums in the march precision (a few sites each), the warp tree in it too, FP64 across warps
  cpx<R> tss[NPH], tbs[NPH], tsb[NPH];
#pragma unroll
  for (int jj = 0; jj < NPH; ++jj) tss[jj] = tbs[jj] = tsb[jj] = mk<R>(0, 0);
#pragma unroll(NPH == 1 ? 2 : 1)
  for (int j = bx * blockDim.x + threadIdx.x; j < g.N; j += nbx * blockDim.x) {
    const int ix = j % g.n[0];
    const int iy = (j / g.n[0]) % g.n[1];
    const int iz = j / (g.n[0] * g.n[1]);
    cpx<R> u[4], v[4], ub[4], vb[4];
    const cpx<R> phu = xmul(xmul(xmul(tfu, tu[ix]), tu[g.n[0] + iy]), tu[g.n[0] + g.n[1] + iz]);
    const cpx<R> phv = xmul(xmul(xmul(tfv, tv[ix]), tv[g.n[0] + iy]), tv[g.n[0] + g.n[1] + iz]);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      u[a] = U[(size_t)a * g.N + j];
      v[a] = V[(size_t)a * g.N + j];
      ub[a] = xmul(tu[nt + a], phu);
      vb[a] = xmul(tv[nt + a], phv);
    }
#pragma unroll
    for (int jj = 0; jj < NPH; ++jj) {
      const cpx<R> ph = xmul(xmul(kp[jj][ix], kp[jj][g.n[0] + iy]), kp[jj][g.n[0] + g.n[1] + iz]);
      cpx<R> av[4], avb[4];
      alpha_eps<R>(eps[jj], v, av);
      alpha_eps<R>(eps[jj], vb, avb);
      cpx<R> ss = mk<R>(0, 0), bs = mk<R>(0, 0), sb = mk<R>(0, 0);
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        ss = xadd(ss, xcdot(u[a], av[a]));
        bs = xadd(bs, xcdot(ub[a], av[a]));
        sb = xadd(sb, xcdot(u[a], avb[a]));
      }
      tss[jj] = xadd(tss[jj], xmul(ss, ph));
      tbs[jj] = xadd(tbs[jj], xmul(bs, ph));
      tsb[jj] = xadd(tsb[jj], xmul(sb, ph));
    }
  }
#pragma unroll
  for (int jj = 0; jj < NPH; ++jj) {
    const cpx<R> ass = warp_sum<R>(tss[jj]), abs_ = warp_sum<R>(tbs[jj]), asb = warp_sum<R>(tsb[jj]);
    if ((threadIdx.x & 31) == 0) {
      red[threadIdx.x >> 5][3 * jj] = cvt<double>(ass);
      red[threadIdx.x >> 5][3 * jj + 1] = cvt<double>(abs_);
      red[threadIdx.x >> 5][3 * jj + 2] = cvt<double>(asb);
    }
  }
  __syncthreads();
  if (threadIdx.x < 3 * nj) {
    const int jj = threadIdx.x / 3, q = threadIdx.x % 3;
    cpx<double> sacc = mk<double>(0, 0);
    for (int wi = 0; wi < 8; ++wi) sacc = xadd(sacc, red[wi][threadIdx.x]);
    const cpx<double>* trow = ptab + 3 * (tab_row + (long)(pi0 + jj) * tab_stride);
    cpx<double>& a = acc[((size_t)(pi0 + jj) * nbx + bx) * 3 + q];
    a = xadd(a, xmul(trow[2], sacc));
  }
}

template <typename R, int NPH>
__global__ void __launch_bounds__(256) k_mdot(const cpx<R>* __restrict__ ys, const cpx<R>* gcplx, const cpx<R>* kph,
                                              const double* photon, GridDesc g, const cpx<double>* __restrict__ ptab,
                                              const MarchClock* clk, int ls, int stage, int tab_stride,
                                              int n_ph, cpx<double>* acc) {
  mdot_body<R, NPH>(ys, gcplx, kph, photon, g, ptab, clk, ls, stage, tab_stride, n_ph, acc, blockIdx.x, blockIdx.y,
                    gridDim.x);
}

// macc[inst][q] = sum_b acc[inst][b][q]: warp q of block inst adds the accumulators
// b = lane, lane + 32, ... in order, then a fixed shuffle tree (deterministic).
__global__ void __launch_bounds__(96) k_mdot_final(const cpx<double>* __restrict__ acc, int nb, cpx<double>* macc) {
  const int inst = blockIdx.x;
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  cpx<double> sacc = mk<double>(0, 0);
  for (int b = lane; b < nb; b += 32) sacc = sacc + acc[((size_t)inst * nb + b) * 3 + q];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sacc.x += __shfl_down_sync(0xffffffffu, sacc.x, off);
    sacc.y += __shfl_down_sync(0xffffffffu, sacc.y, off);
  }
  if (lane == 0) macc[3 * inst + q] = sacc;
}

// ---------------------------------------------------------------- partial-integration form (Sec. IV, Eqs. 28-33)
// The integrand of Eq. 33 and its analogues for (back, scat) and (scat, back), written with the grid
// transform psi~(kappa) and the energy projectors P_sigma of Eq. 23.  The time derivative of the split
// parts P_sigma psi~ e^{i sigma E t} is P_sigma F[Z] with Z = -i V (psi_s + psi_b) (Eq. 6), so per
// stage the march needs F[psi_s] and F[Z] of both waves on every grid mode (ss) and F[Z] at one
// off-grid momentum per wave (bs: V wave at p - k, sb: U wave at k - q).

// Per wave and axis: exp(-i kappa_a x_a) on the grid coordinates (trivial axes: 1), kappa = the wave's
// direct-transform momentum (3 doubles per wave).
template <typename R>
__global__ void k_f2_dtables(const double* wave_k, GridDesc g, int n_waves, cpx<R>* dph) {
  const int nt = g.n[0] + g.n[1] + g.n[2];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_waves * nt; i += gridDim.x * blockDim.x) {
    const int wv = i / nt;
    int j = i % nt, axis = 0;
    while (j >= g.n[axis]) { j -= g.n[axis]; ++axis; }
    const double xc = g.n[axis] > 1 ? g.x0[axis] + j * g.dx[axis] : 0.0;
    double sn, cs;
    sincos(-wave_k[3 * wv + axis] * xc, &sn, &cs);
    dph[i] = mk<R>((R)cs, (R)sn);
  }
}

// Parameters of one mode-sum table: the photon's mode shift per axis, the fixed momenta of U and V
// along trivial axes, and k0.
struct F2Table {
  int shift[3];
  int pad;
  double Ku[3], Kv[3], k0;
};

// Per table and U grid mode j (V mode j - shift, periodic): 1 / Omega_{sigma sigma'} for
// (sigma, sigma') = (+,+), (+,-), (-,+), (-,-), Omega = sigma E_u - sigma' E_v - k0, in FP64 and
// rounded once.  (On the raw transforms the pair's grid-sum factor e^{i(kappa_v + k - kappa_u).x0}
// and the two origin phases combine into e^{i k.x0} for every pair, wrapped or not; the finalize
// kernel applies it.)
template <typename R>
__global__ void k_f2_omega_table(const F2Table* tabs, GridDesc g, int n_tab, R* omt) {
  const long total = (long)n_tab * g.N;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
    const F2Table& T = tabs[e / g.N];
    const int j = (int)(e % g.N);
    const int id[3] = {j % g.n[0], (j / g.n[0]) % g.n[1], j / (g.n[0] * g.n[1])};
    double ku[3], kv[3];
    for (int a = 0; a < 3; ++a) {
      const int jv = ((id[a] - T.shift[a]) % g.n[a] + g.n[a]) % g.n[a];
      ku[a] = kappa_of(id[a], g.n[a], g.L[a], T.Ku[a]);
      kv[a] = kappa_of(jv, g.n[a], g.L[a], T.Kv[a]);
    }
    const double eu = energy3(ku), ev = energy3(kv);
    R* o = omt + 4 * e;
    o[0] = (R)(1.0 / (eu - ev - T.k0));
    o[1] = (R)(1.0 / (eu + ev - T.k0));
    o[2] = (R)(1.0 / (-eu - ev - T.k0));
    o[3] = (R)(1.0 / (-eu + ev - T.k0));
  }
}

// x lines of `rows` grid rows of wave f = 2 inst + (0: U, 1: V) at a weighted stage:
// Z = -i V (Y + psi_b) of the stage value Y (from ys; the local term of the right-hand side,
// evaluated as in k_first) x-transformed into Zspec[f], and with do_y also Y into Yspec[f] (grids
// without a y or z pass; otherwise the right-hand side's pass writes the transform of Y); and
// the block's part of sum_x exp(-i kappa.x) Z(x) (the wave's direct transform), which
// trow[w] (w_i and its time phase) times adds to the block's own FP64 accumulators
// dpart[f][block][4] (no other block touches them: the sum is deterministic).
template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 2) k_f2_x(StageArgs<R> A, const cpx<R>* __restrict__ ys, cpx<R>* __restrict__ Yspec,
                                              cpx<R>* __restrict__ Zspec, int do_y, const cpx<R>* __restrict__ dph,
                                              const cpx<double>* __restrict__ ptab, int tab_stride, int stage,
                                              cpx<double>* dpart, int rows, int ld) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* buf = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* buf2 = buf + 4 * rows * ld;
  __shared__ R s_ft[64];  // field time factor per row, computed in FP64 and rounded once
  __shared__ cpx<R> s_tf;
  __shared__ cpx<double> red[8][4];
  const int f = blockIdx.y;
  const int inst = f >> 1, w = f & 1;
  const int row0 = blockIdx.x * rows;
  const int nx = A.g.n[0], ny = A.g.n[1], nz = A.g.n[2];
  const int N = A.g.N;
  const size_t fo = (size_t)f * 4 * N;
  const size_t cs = (size_t)N;
  const FieldDesc* F = A.fd + f;
  const double tst = stage_time(A);
  for (int j = threadIdx.x; j < rows; j += blockDim.x) {
    const int iy = (row0 + j) % ny;
    const double yc = ny > 1 ? A.g.x0[1] + iy * A.g.dx[1] : 0.0;
    s_ft[j] = (R)field_time_factor(*F, tst, yc);
  }
  if (threadIdx.x == 0) {
    double sn, c;
    sincos(F->tsign * F->e0 * tst, &sn, &c);
    s_tf = mk<R>((R)c, (R)sn);
  }
  __syncthreads();
  const int nt = nx + ny + nz;
  const R* gx = A.greal + (size_t)f * nt;
  const R* gy = gx + nx;
  const R* gz = gy + ny;
  const cpx<R>* ex = A.gcplx + (size_t)f * (nt + 4);
  const cpx<R>* ey = ex + nx;
  const cpx<R>* ez = ey + ny;
  const cpx<R>* wsp = ez + nz;
  const cpx<R>* dx = dph + (size_t)f * nt;
  const int acomp = F->acomp;
  const int per = rows * nx;
  cpx<R>* sy = Yspec + fo;
  cpx<R>* sz = Zspec + fo;
  cpx<R> dsum[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) dsum[c] = mk<R>(0, 0);
  for (int part = do_y ? 0 : 1; part < 2; ++part) {
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int j = e / nx;
      const int x = e - j * nx;
      const int row = row0 + j;
      cpx<R> v[4];
      if (row < A.nrows) {
        const size_t gi = fo + (size_t)row * nx + x;
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = ys[gi + c * cs];
        if (part == 1) {
          const int iy = row % ny, iz = row / ny;
          const R a = s_ft[j] * gx[x] * gy[iy] * gz[iz];
          const cpx<R> ph = s_tf * ex[x] * ey[iy] * ez[iz];
          cpx<R> phi[4], vz[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) phi[c] = v[c] + wsp[c] * ph;
          apply_v<R>(acomp, a, phi, vz);
          const cpx<R> dp = dx[x] * dx[nx + iy] * dx[nx + ny + iz];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            v[c] = mul_mi(vz[c]);
            dsum[c] = dsum[c] + v[c] * dp;
          }
        }
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) v[c] = mk<R>(0, 0);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) buf[(c * rows + j) * ld + pad32(x)] = v[c];
    }
    __syncthreads();
    cpx<R>* res = fft_pp<R>(buf, buf2, ld, 4 * rows, A.plan[0], false, A.tw[0]);
    cpx<R>* dst = part == 0 ? sy : sz;
    for (int e = threadIdx.x; e < per; e += blockDim.x) {
      const int j = e / nx;
      const int x = e - j * nx;
      const int row = row0 + j;
      if (row < A.nrows) {
        const size_t gi = (size_t)row * nx + x;
#pragma unroll
        for (int c = 0; c < 4; ++c) dst[gi + c * cs] = res[(c * rows + j) * ld + pad32(x)];
      }
    }
    __syncthreads();
  }
  // block sum of the direct transform (warp trees in the march precision, FP64 across warps)
  cpx<R> ds[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) ds[c] = warp_sum<R>(dsum[c]);
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int c = 0; c < 4; ++c) red[threadIdx.x >> 5][c] = cvt<double>(ds[c]);
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    const long tab_row = (long)(A.clk->step + A.ls) * 7 + stage;
    const cpx<double> wt = ptab[3 * (tab_row + (long)inst * tab_stride) + w];
    cpx<double> sacc = mk<double>(0, 0);
    for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) sacc = sacc + red[wi][threadIdx.x];
    cpx<double>& a = dpart[((size_t)f * gridDim.x + blockIdx.x) * 4 + threadIdx.x];
    a = a + wt * sacc;
  }
}

// o = P_+(kappa) x = (x + H0(kappa) x / E) / 2, the positive-energy part (evolves as e^{-iEt}).
template <typename R>
__device__ __forceinline__ void proj_plus(const R* kk, R inv_e, const cpx<R>* x, cpx<R>* o) {
  cpx<R> hx[4];
  alpha_eps<R>(kk, x, hx);
  const R hh = (R)0.5 * inv_e;
  o[0] = (R)0.5 * x[0] + hh * (hx[0] + x[0]);
  o[1] = (R)0.5 * x[1] + hh * (hx[1] + x[1]);
  o[2] = (R)0.5 * x[2] + hh * (hx[2] - x[2]);
  o[3] = (R)0.5 * x[3] + hh * (hx[3] - x[3]);
}

// sum_a conj(x_a) (alpha.eps y)_a
template <typename R>
__device__ __forceinline__ cpx<R> form_ae(const cpx<R>* x, const cpx<R>* aey) {
  cpx<R> d = cdot(x[0], aey[0]);
#pragma unroll
  for (int a = 1; a < 4; ++a) d = d + cdot(x[a], aey[a]);
  return d;
}

// The mode sum of the (scat, scat) integrand at one weighted stage, on the raw transforms Yspec, Zspec
// of the waves (no cell factor, no origin phase):
//   sum_j sum_{sigma,sigma'} 1/Omega [ (P_s Zu~)^+ (alpha.eps) P_s' Yv~ + (P_s Yu~)^+ (alpha.eps) P_s' Zv~ ]
// with U quantities at mode j and V quantities at mode j - shift.  Block (b, inst) adds trow[2]
// (w_i e^{-i k0 t}) times its part to its own accumulator sspart[inst][b].
// f2i per instance: shift[3], table index.
template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 1) k_f2_ss(const cpx<R>* __restrict__ Yspec, const cpx<R>* __restrict__ Zspec,
                                               GridDesc g, const FieldDesc* fd,
                                               const double* photon, const int* __restrict__ f2i,
                                               const R* __restrict__ omt, const cpx<double>* __restrict__ ptab,
                                               const MarchClock* clk, int ls, int stage, int tab_stride,
                                               cpx<double>* sspart) {
  __shared__ cpx<double> red[8];
  const int inst = blockIdx.y;
  const int N = g.N;
  const int shift[3] = {f2i[4 * inst], f2i[4 * inst + 1], f2i[4 * inst + 2]};
  const R* om = omt + (size_t)f2i[4 * inst + 3] * 4 * N;
  const FieldDesc& FU = fd[2 * inst];
  const FieldDesc& FV = fd[2 * inst + 1];
  R eps[3];
  for (int a = 0; a < 3; ++a) eps[a] = (R)photon[6 * inst + 3 + a];
  const cpx<R>* Yu = Yspec + (size_t)(2 * inst) * 4 * N;
  const cpx<R>* Yv = Yu + (size_t)4 * N;
  const cpx<R>* Zu = Zspec + (size_t)(2 * inst) * 4 * N;
  const cpx<R>* Zv = Zu + (size_t)4 * N;
  // mode spacing 2 pi / L per axis (the mode index times it is kappa; trivial axes: fixed K)
  R du[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) du[a] = (R)(6.283185307179586476925286766559 / g.L[a]);
  cpx<R> tacc = mk<R>(0, 0);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N; j += gridDim.x * blockDim.x) {
    const int id[3] = {j % g.n[0], (j / g.n[0]) % g.n[1], j / (g.n[0] * g.n[1])};
    int jv[3];
    R ku[3], kv[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int n = g.n[a];
      jv[a] = id[a] - shift[a];
      if (jv[a] < 0) jv[a] += n;
      if (jv[a] >= n) jv[a] -= n;
      const int fu = id[a] < (n + 1) / 2 ? id[a] : id[a] - n;
      const int fv = jv[a] < (n + 1) / 2 ? jv[a] : jv[a] - n;
      ku[a] = n > 1 ? du[a] * (R)fu : (R)FU.K[a];
      kv[a] = n > 1 ? du[a] * (R)fv : (R)FV.K[a];
    }
    const int j2 = (jv[2] * g.n[1] + jv[1]) * g.n[0] + jv[0];
    const R ieu = (R)1 / sqrt((R)1 + ku[0] * ku[0] + ku[1] * ku[1] + ku[2] * ku[2]);
    const R iev = (R)1 / sqrt((R)1 + kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2]);
    cpx<R> y[4], z[4], ap[4], am[4], dap[4], dam[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      y[c] = Yu[(size_t)c * N + j];
      z[c] = Zu[(size_t)c * N + j];
    }
    proj_plus<R>(ku, ieu, y, ap);
    proj_plus<R>(ku, ieu, z, dap);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      am[c] = y[c] - ap[c];
      dam[c] = z[c] - dap[c];
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      y[c] = Yv[(size_t)c * N + j2];
      z[c] = Zv[(size_t)c * N + j2];
    }
    cpx<R> bp[4], bm[4], dbp[4], dbm[4], t1[4], t2[4];
    proj_plus<R>(kv, iev, y, t1);
    proj_plus<R>(kv, iev, z, t2);
    alpha_eps<R>(eps, t1, bp);
    alpha_eps<R>(eps, t2, dbp);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      t1[c] = y[c] - t1[c];
      t2[c] = z[c] - t2[c];
    }
    alpha_eps<R>(eps, t1, bm);
    alpha_eps<R>(eps, t2, dbm);
    const R* o = om + 4 * (size_t)j;
    const R opp = o[0], opm = o[1], omp = o[2], omm = o[3];
    tacc = tacc + opp * (form_ae<R>(dap, bp) + form_ae<R>(ap, dbp));
    tacc = tacc + opm * (form_ae<R>(dap, bm) + form_ae<R>(ap, dbm));
    tacc = tacc + omp * (form_ae<R>(dam, bp) + form_ae<R>(am, dbp));
    tacc = tacc + omm * (form_ae<R>(dam, bm) + form_ae<R>(am, dbm));
  }
  const cpx<R> s = warp_sum<R>(tacc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cvt<double>(s);
  __syncthreads();
  if (threadIdx.x == 0) {
    const long tab_row = (long)(clk->step + ls) * 7 + stage;
    const cpx<double> wt = ptab[3 * (tab_row + (long)inst * tab_stride) + 2];
    cpx<double> sacc = mk<double>(0, 0);
    for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) sacc = sacc + red[wi];
    cpx<double>& a = sspart[(size_t)inst * gridDim.x + blockIdx.x];
    a = a + wt * sacc;
  }
}

// macc[inst] = (ss, D_U[4], D_V[4]): warp 0 sums the mode-sum accumulators of the instance, warps
// 1-4 the U wave's direct transform components, warps 5-8 the V wave's, each in a fixed order.
__global__ void __launch_bounds__(288) k_f2_final(const cpx<double>* __restrict__ sspart, int nbs,
                                                  const cpx<double>* __restrict__ dpart, int nbx,
                                                  cpx<double>* macc) {
  const int inst = blockIdx.x;
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  cpx<double> sacc = mk<double>(0, 0);
  if (q == 0) {
    for (int b = lane; b < nbs; b += 32) sacc = sacc + sspart[(size_t)inst * nbs + b];
  } else {
    const int wv = 2 * inst + (q - 1) / 4, c = (q - 1) % 4;
    for (int b = lane; b < nbx; b += 32) sacc = sacc + dpart[((size_t)wv * nbx + b) * 4 + c];
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sacc.x += __shfl_down_sync(0xffffffffu, sacc.x, off);
    sacc.y += __shfl_down_sync(0xffffffffu, sacc.y, off);
  }
  if (lane == 0) macc[9 * inst + q] = sacc;
}

// Buffers and launch shapes of the partial-integration integrand.
template <typename R>
struct F2Plan {
  cpx<R>* Yspec = nullptr;   // [2 n_inst][4][N]: transforms of the stage values Y of both waves
  cpx<R>* Zspec = nullptr;   // [2 n_inst][4][N]: transforms of Z = -i V (Y + psi_b)
  int has_mid = 0;           // a y or z pass exists (it writes Yspec)
  cpx<R>* dph = nullptr;     // [2 n_inst][nx + ny + nz]: direct-transform phases per wave
  int* f2i = nullptr;        // [n_inst][4]: photon mode shift, table index
  R* omt = nullptr;          // [tables][N][4]: rho / Omega
  cpx<double>* dpart = nullptr;   // [2 n_inst][nbx][4]
  cpx<double>* sspart = nullptr;  // [n_inst][nbs]
  int n_inst = 0, nbx = 0, nbs = 0, rows = 0, ld = 0, xthr = 256;
  size_t smem_x = 0;
};

template <typename R>
static swf_status f2_prepare(swf_ctx* ctx, const GridDesc& g, int n_inst, const FieldDesc* fd_host,
                             const double* photon_host, const double* wave_k_host,
                             F2Plan<R>* p, cudaStream_t st) {
  static bool attr_done[64] = {false};
  const int dv = dev_slot();
  cudaError_t e;
  if (!attr_done[dv]) {
    e = cudaFuncSetAttribute(k_f2_x<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmem);
    if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(k_f2_x)");
    attr_done[dv] = true;
  }
  const int nx = g.n[0];
  const int nrows = g.n[1] * g.n[2];
  const int nt = g.n[0] + g.n[1] + g.n[2];
  p->n_inst = n_inst;
  // a fixed shape (not the tuned one of the right-hand side's x passes): the block's rows and
  // threads decide the order of the direct-transform sums, which must not depend on timing
  p->rows = x_rows<R>(nx, nrows, 2 * n_inst);
  p->xthr = kThreads;
  if (p->rows < 1) {
    set_error("partial-integration integrand: an x line does not fit shared memory");
    return SWF_EUNSUPPORTED;
  }
  p->ld = padded_len(nx);
  p->smem_x = (size_t)2 * 4 * p->rows * p->ld * sizeof(cpx<R>);
  p->nbx = (nrows + p->rows - 1) / p->rows;
  // one mode per thread where the grid allows (the gathers of the V modes are latency-bound)
  p->nbs = std::max(1, std::min((g.N + 255) / 256, (32 * sm_count() + n_inst - 1) / n_inst));
  // mode-sum tables, shared by instances with the same photon shift, trivial-axis momenta and k0
  std::vector<int> info(4 * (size_t)n_inst);
  std::vector<F2Table> tabs;
  std::map<std::vector<double>, int> seen;
  for (int i = 0; i < n_inst; ++i) {
    F2Table T;
    std::memset(&T, 0, sizeof T);
    const double* k = photon_host + 6 * i;
    for (int a = 0; a < 3; ++a) {
      T.shift[a] = g.n[a] > 1 ? (int)std::lround(k[a] * g.L[a] / 6.283185307179586476925286766559) : 0;
      T.Ku[a] = fd_host[2 * i].K[a];
      T.Kv[a] = fd_host[2 * i + 1].K[a];
    }
    T.k0 = std::sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    const std::vector<double> key = {(double)T.shift[0], (double)T.shift[1], (double)T.shift[2], T.Ku[0], T.Ku[1],
                                     T.Ku[2], T.Kv[0], T.Kv[1], T.Kv[2], T.k0};
    auto it = seen.find(key);
    int id;
    if (it == seen.end()) {
      id = (int)tabs.size();
      seen[key] = id;
      tabs.push_back(T);
    } else {
      id = it->second;
    }
    for (int a = 0; a < 3; ++a) info[4 * i + a] = T.shift[a];
    info[4 * i + 3] = id;
  }
  const int n_tab = (int)tabs.size();
  constexpr size_t esz = sizeof(cpx<R>);
  void *pY, *pZ, *pdph, *pinfo, *ptabs, *pomt, *pdp, *pss, *pwk;
  swf_status s;
  if ((s = ws_get(ctx, "bw2.yspec", (size_t)2 * n_inst * 4 * g.N * esz, &pY)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bw2.zspec", (size_t)2 * n_inst * 4 * g.N * esz, &pZ)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bw2.dph", (size_t)2 * n_inst * nt * esz, &pdph)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bw2.wavek", sizeof(double) * 6 * (size_t)n_inst, &pwk)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bw2.info", sizeof(int) * 4 * (size_t)n_inst, &pinfo)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bw2.tabs", sizeof(F2Table) * (size_t)n_tab, &ptabs)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bw2.omega", sizeof(R) * 4 * (size_t)n_tab * g.N, &pomt)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bw2.dpart", sizeof(cpx<double>) * 4 * (size_t)2 * n_inst * p->nbx, &pdp)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bw2.sspart", sizeof(cpx<double>) * (size_t)n_inst * p->nbs, &pss)) != SWF_OK) return s;
  p->Yspec = (cpx<R>*)pY;
  p->Zspec = (cpx<R>*)pZ;
  p->has_mid = (g.n[1] > 1 || g.n[2] > 1) ? 1 : 0;
  p->dph = (cpx<R>*)pdph;
  p->f2i = (int*)pinfo;
  p->omt = (R*)pomt;
  p->dpart = (cpx<double>*)pdp;
  p->sspart = (cpx<double>*)pss;
  if ((e = cudaMemcpyAsync(pwk, wave_k_host, sizeof(double) * 6 * n_inst, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(pinfo, info.data(), sizeof(int) * info.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(ptabs, tabs.data(), sizeof(F2Table) * tabs.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cuda_status(e, "upload partial-integration tables");
  if ((e = cudaMemsetAsync(pdp, 0, sizeof(cpx<double>) * 4 * (size_t)2 * n_inst * p->nbx, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(pss, 0, sizeof(cpx<double>) * (size_t)n_inst * p->nbs, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(pY, 0, (size_t)2 * n_inst * 4 * g.N * esz, st)) != cudaSuccess)
    return cuda_status(e, "memset partial-integration accumulators");
  {
    ProfScope ps(ctx, "k_f2_dtables", st);
    k_f2_dtables<R><<<(2 * n_inst * nt + 127) / 128, 128, 0, st>>>((const double*)pwk, g, 2 * n_inst, p->dph);
  }
  {
    const long total = (long)n_tab * g.N;
    ProfScope ps(ctx, "k_f2_omega_table", st);
    k_f2_omega_table<R><<<(int)std::min((total + 255) / 256, 8192L), 256, 0, st>>>((const F2Table*)ptabs, g, n_tab,
                                                                                   p->omt);
  }
  // the host tables above are temporaries
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "partial-integration tables");
  return SWF_OK;
}

// One evaluation of the partial-integration integrand at stage `stage` of step (clock step + ls), on
// the stage values ys of all waves: the x transform of Z (and of Y on grids without a y or z pass;
// otherwise the right-hand side's pass has written F[Y]) with the direct transforms, the forward y
// (and z) transforms of Z, then the mode sum.
template <typename R>
static swf_status f2_integrand(swf_ctx* ctx, const StageArgs<R>& A, const F2Plan<R>& p, const cpx<R>* ys,
                               const double* photon_dev, const cpx<double>* ptab, int tab_stride, int ls, int stage,
                               cudaStream_t st) {
  const GridDesc& g = A.g;
  const int G = p.n_inst;
  StageArgs<R> B = A;
  B.ls = ls;
  B.c = DP_C[stage];
  {
    ProfScope ps(ctx, "k_f2_x", st);
    k_f2_x<R><<<dim3(p.nbx, 2 * G), p.xthr, p.smem_x, st>>>(B, ys, p.Yspec, p.Zspec, p.has_mid ? 0 : 1, p.dph,
                                                             ptab, tab_stride, stage, p.dpart, p.rows, p.ld);
  }
  StageArgs<R> C = A;
  C.T = p.Zspec;
  C.yspec = nullptr;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  for (int axis = 1; axis <= 2; ++axis) {
    if (g.n[axis] <= 1) continue;
    const int other = axis == 1 ? nz : ny;
    const MidShape ms = mid_shape<R>(g.n[axis], nx, (long)other * 2 * G);
    const int ntx = (nx + (1 << ms.lgtx) - 1) >> ms.lgtx;
    ProfScope ps(ctx, "k_mid", st);
    k_mid<R><<<dim3(ntx * other, 2 * G), kThreads, ms.smem, st>>>(C, axis, ms.lgtx, ms.ld, 1, 0, 0);
  }
  {
    ProfScope ps(ctx, "k_f2_ss", st);
    k_f2_ss<R><<<dim3(p.nbs, G), kThreads, 0, st>>>(p.Yspec, p.Zspec, g, A.fd, photon_dev, p.f2i, p.omt, ptab, A.clk,
                                                    ls, stage, tab_stride, p.sspart);
  }
  return SWF_OK;
}

template <typename R>
static swf_status march_bw_impl(swf_ctx* ctx, const GridDesc& g, double t_in, double t_out, int n_steps, int n_inst,
                                const FieldDesc* fd_host, const double* photon_host, void* psi_out, double2* macc,
                                cudaStream_t st, int form, const double* wave_k_host, int n_ph) {
  const int F = 2 * n_inst;
  const int NP = n_inst * n_ph;  // photon-instances: photon j of instance i is i n_ph + j
  StageArgs<R> A;
  swf_status s = prepare_args<R>(ctx, g, F, fd_host, &A, "bw", st);
  if (s != SWF_OK) return s;
  const size_t state = (size_t)F * 4 * g.N * sizeof(cpx<R>);
  const int nt = g.n[0] + g.n[1] + g.n[2];
  void *py, *pT, *pys, *pk[7], *pph, *pkph;
  if ((s = ws_get(ctx, "march.y", state, &py)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "march.T", state, &pT)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bw.ystage", state, &pys)) != SWF_OK) return s;
  for (int i = 0; i < 7; ++i) {
    char nm[32];
    std::snprintf(nm, sizeof nm, "march.k%d", i);
    if ((s = ws_get(ctx, nm, state, &pk[i])) != SWF_OK) return s;
  }
  if ((s = ws_get(ctx, "bw.photon", sizeof(double) * 6 * NP, &pph)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bw.kph", sizeof(cpx<R>) * NP * nt, &pkph)) != SWF_OK) return s;
  // blocks per instance of the M-dot reduction: about four waves of the GPU in total, at least
  // 1024 sites per block (the same split for every photon count, so a photon of a scan sums
  // exactly as a solve of that photon alone); photons per block: 1, or 4 (8 in complex64) for
  // scans, which then read U and V once per site for the block's photons
  const int nph_blk = n_ph == 1 ? 1 : (sizeof(R) == 4 && n_ph > 4 ? 8 : 4);
  const int nchunk = (n_ph + nph_blk - 1) / nph_blk;
  const int nb = std::max(1, std::min((g.N + 1023) / 1024, (4 * sm_count() + n_inst - 1) / n_inst));
  void* ptab;
  if ((s = ws_get(ctx, "bw.phase_table", sizeof(cpx<double>) * 3 * 7 * (size_t)n_steps * NP, &ptab)) != SWF_OK)
    return s;
  void* ppart;
  if ((s = ws_get(ctx, "bw.mpart", sizeof(cpx<double>) * 3 * (size_t)nb * NP, &ppart)) != SWF_OK) return s;
  cudaError_t e = cudaMemcpyAsync(pph, photon_host, sizeof(double) * 6 * NP, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "upload photon table");
  {
    ProfScope ps(ctx, "k_photon_tables", st);
    k_photon_tables<R><<<(NP * nt + 127) / 128, 128, 0, st>>>((const double*)pph, g, NP, (cpx<R>*)pkph);
  }
  {
    const long total = (long)NP * n_steps * 7;
    ProfScope ps(ctx, "k_bw_phase_table", st);
    k_bw_phase_table<<<(int)std::min((total + 127) / 128, 4096L), 128, 0, st>>>(
        A.fd, (const double*)pph, NP, n_ph, n_steps, t_out, (t_in - t_out) / n_steps, g.dx[0] * g.dx[1] * g.dx[2],
        form, (cpx<double>*)ptab);
  }
  if ((e = cudaMemsetAsync(py, 0, state, st)) != cudaSuccess) return cuda_status(e, "memset state");
  if ((e = cudaMemsetAsync(ppart, 0, sizeof(cpx<double>) * 3 * (size_t)nb * NP, st)) != cudaSuccess)
    return cuda_status(e, "memset M accumulators");
  A.y = (cpx<R>*)py;
  A.T = (cpx<R>*)pT;
  if ((s = state_low_part<R>(ctx, "march.ylo", state, &A, st)) != SWF_OK) return s;
  {
    StageArgs<R> B = A;  // shapes by timing, as in the plain march
    B.nterm = 6;
    for (int q = 0; q < 6; ++q) {
      B.kin[q] = (const cpx<R>*)pk[q + 1];
      B.coef[q] = 0.0;
    }
    B.write_y = 0;
    B.ystage = nullptr;
    B.kout = (cpx<R>*)pk[0];
    B.t = t_out;
    if ((s = autotune_eval<R>(ctx, B, F, st)) != SWF_OK) return s;
  }
  F2Plan<R> p2;
  if (form == 2 && (s = f2_prepare<R>(ctx, g, n_inst, fd_host, photon_host, wave_k_host, &p2, st)) != SWF_OK)
    return s;
  int slot[7] = {0, 1, 2, 3, 4, 5, 6};
  const double h = (t_in - t_out) / n_steps;
  void* pclk = nullptr;
  if ((s = ws_get(ctx, "march.clock", sizeof(MarchClock), &pclk)) != SWF_OK) return s;
  MarchClock* clk = (MarchClock*)pclk;
  k_clock_set<<<1, 1, 0, st>>>(clk, t_out, h);
  A.clk = clk;
  A.nterm = 0;
  A.write_y = 0;
  A.kout = (cpx<R>*)pk[slot[0]];
  A.ls = 0;
  A.c = 0.0;
  A.ystage = nullptr;  // the integrand of Eq. 17 vanishes at psi_s(t_out) = 0
  // evaluations chain through k_last_first as in march_impl (the integrands read only the stage
  // value and the transforms written by the forward passes, never T or the k slots)
  const bool chain = !(g.n[1] == 1 && g.n[2] == 1);
  if ((s = chain ? launch_eval_open<R>(ctx, A, F, st) : launch_eval<R>(ctx, A, F, st)) != SWF_OK) return s;
  StageArgs<R> open = A;
  // the partial-integration integrand does not (its source term is V psi_b): stage value y = 0
  if (form == 2 && (s = f2_integrand<R>(ctx, A, p2, (const cpx<R>*)py, (const double*)pph, (const cpx<double>*)ptab,
                                        7 * n_steps, 0, 0, st)) != SWF_OK)
    return s;
  auto step = [&](int ls) -> swf_status {
    for (int i = 1; i < 7; ++i) {
      int ntm = 0;
      for (int j = 0; j < i; ++j) {
        if (DP_A[i][j] == 0.0) continue;
        A.kin[ntm] = (const cpx<R>*)pk[slot[j]];
        A.coef[ntm] = h * DP_A[i][j];
        ++ntm;
      }
      A.nterm = ntm;
      A.write_y = (i == 6);
      A.kout = (cpx<R>*)pk[slot[i]];
      A.ls = ls;
      A.c = DP_C[i];
      // stage values with a quadrature weight: b_{i+1} for i = 2..5 and, for the new state
      // (i = 6), b_1 of the next step (the phase table holds 0 there on the last step, so every
      // step launches the same kernels)
      const bool weighted = i >= 2;
      A.ystage = weighted ? (cpx<R>*)pys : nullptr;
      A.yspec = (weighted && form == 2) ? p2.Yspec : nullptr;  // the y or z pass writes F[Y] (if there is one)
      swf_status r = chain ? launch_eval_chain<R>(ctx, open, A, F, st) : launch_eval<R>(ctx, A, F, st);
      if (r != SWF_OK) return r;
      open = A;
      if (weighted && form == 2) {
        if ((r = f2_integrand<R>(ctx, A, p2, (const cpx<R>*)pys, (const double*)pph, (const cpx<double>*)ptab,
                                 7 * n_steps, ls, i, st)) != SWF_OK)
          return r;
      } else if (weighted) {
        ProfScope ps(ctx, "k_mdot", st);
        const cpx<R>* ysc = (const cpx<R>*)pys;
        const cpx<R>* kpc = (const cpx<R>*)pkph;
        const cpx<double>* tb = (const cpx<double>*)ptab;
        cpx<double>* pa = (cpx<double>*)ppart;
        const dim3 grid(nb, n_inst * nchunk);
        if (nph_blk == 1)
          k_mdot<R, 1><<<grid, 256, 0, st>>>(ysc, A.gcplx, kpc, (const double*)pph, g, tb, clk, ls, i, 7 * n_steps,
                                             n_ph, pa);
        else if (nph_blk == 4)
          k_mdot<R, 4><<<grid, 256, 0, st>>>(ysc, A.gcplx, kpc, (const double*)pph, g, tb, clk, ls, i, 7 * n_steps,
                                             n_ph, pa);
        else
          k_mdot<R, 8><<<grid, 256, 0, st>>>(ysc, A.gcplx, kpc, (const double*)pph, g, tb, clk, ls, i, 7 * n_steps,
                                             n_ph, pa);
      }
    }
    std::swap(slot[0], slot[6]);
    return SWF_OK;
  };
  s = run_step_pairs(ctx, st, n_steps / 2, clk, [&]() -> swf_status {
    swf_status r = step(0);
    return r == SWF_OK ? step(1) : r;
  });
  if (s != SWF_OK) return s;
  if (n_steps % 2 && (s = step(0)) != SWF_OK) return s;
  if (chain && (s = launch_eval_close<R>(ctx, open, F, st)) != SWF_OK) return s;
  if (form == 2) {
    ProfScope ps(ctx, "k_f2_final", st);
    k_f2_final<<<n_inst, 288, 0, st>>>(p2.sspart, p2.nbs, p2.dpart, p2.nbx, (cpx<double>*)macc);
  } else {
    ProfScope ps(ctx, "k_mdot_final", st);
    k_mdot_final<<<NP, 96, 0, st>>>((const cpx<double>*)ppart, nb, (cpx<double>*)macc);
  }
  e = cudaMemcpyAsync(psi_out, py, state, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "copy psi(t_in)");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "Breit-Wheeler march kernels");
  return SWF_OK;
}

swf_status march_bw(swf_ctx* ctx, const GridDesc& g, double t_in, double t_out, int n_steps, int n_inst,
                    const FieldDesc* fd_host, const double* photon_host, swf_precision prec, void* psi_out,
                    double2* macc, cudaStream_t st, int form, const double* wave_k_host, int n_ph) {
  if (form == 2 && (!wave_k_host || n_ph != 1)) {
    set_error("march_bw: the partial-integration form needs the direct-transform momenta and one photon per instance");
    return SWF_EINVAL;
  }
  if (n_ph < 1) {
    set_error("march_bw: at least one photon per instance");
    return SWF_EINVAL;
  }
  if (prec == SWF_C64)
    return march_bw_impl<float>(ctx, g, t_in, t_out, n_steps, n_inst, fd_host, photon_host, psi_out, macc, st, form,
                                wave_k_host, n_ph);
  return march_bw_impl<double>(ctx, g, t_in, t_out, n_steps, n_inst, fd_host, photon_host, psi_out, macc, st, form,
                               wave_k_host, n_ph);
}

// ---------------------------------------------------------------- step-size-controlled Breit-Wheeler march
// Per attempt and photon-instance: the stage rows of the integrand's phase table from the
// controller's t and h (stage i at t + c_i h): the U and V background time phases and the
// quadrature factor h b_{i+1} dx^d e^{-i k0 t} (stage 0 is the accepted state y_n, stage 6 the
// new state, whose weight b_7 is zero).  rows [inst][7][3].
__global__ void k_bw_attempt_rows(const FieldDesc* fd, const double* photon, const StepControl* ctl, double cell,
                                  cpx<double>* rows) {
  const int inst = blockIdx.x, i = threadIdx.x;
  if (i >= 7 || ctl->done) return;
  const double DPc[7] = {0.0, 0.2, 0.3, 0.8, 8.0 / 9.0, 1.0, 1.0};
  const double DPb[7] = {35.0 / 384, 0.0, 500.0 / 1113, 125.0 / 192, -2187.0 / 6784, 11.0 / 84, 0.0};
  const double t = ctl->t + DPc[i] * ctl->h;
  const double w = ctl->h * DPb[i];
  const FieldDesc& FU = fd[2 * inst];
  const FieldDesc& FV = fd[2 * inst + 1];
  const double* k = photon + 6 * inst;
  const double k0 = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
  double sn, cs;
  cpx<double>* r = rows + 3 * (7 * (size_t)inst + i);
  sincos(FU.tsign * FU.e0 * t, &sn, &cs);
  r[0] = mk<double>(cs, sn);
  sincos(FV.tsign * FV.e0 * t, &sn, &cs);
  r[1] = mk<double>(cs, sn);
  sincos(-k0 * t, &sn, &cs);
  r[2] = mk<double>(w * cell * cs, w * cell * sn);
}

// After an accepted attempt: the attempt's integrand sums join the march's.
__global__ void k_mdot_commit(const StepControl* ctl, const cpx<double>* __restrict__ tryacc, cpx<double>* acc,
                              size_t n) {
  if (!ctl->ok) return;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    acc[i] = acc[i] + tryacc[i];
}

// The Breit-Wheeler march (U and V of every instance, the integrand of Eq. 17 appended) with
// step-size control: one controller for all 2 n_inst waves (the error norm is the largest of
// theirs), each attempt one graph replay as in march_adaptive_impl.  The integrand is summed per
// attempt and committed only when the step is accepted.  macc [n_inst][3] as march_bw's form 1.
template <typename R>
static swf_status march_bw_adaptive_impl(swf_ctx* ctx, const GridDesc& g, double t_in, double t_out, double h0,
                                         int max_attempts, int n_inst, const FieldDesc* fd_host,
                                         const double* photon_host, void* psi_out, double2* macc, cudaStream_t st) {
  const int F = 2 * n_inst;
  StageArgs<R> A;
  swf_status s = prepare_args<R>(ctx, g, F, fd_host, &A, "bw", st);
  if (s != SWF_OK) return s;
  const size_t per_field = (size_t)4 * g.N;
  const size_t state = (size_t)F * per_field * sizeof(cpx<R>);
  const int nt = g.n[0] + g.n[1] + g.n[2];
  void *py, *pyn, *pT, *pys, *pk[7], *pctl, *ppart, *pph, *pkph, *prow, *pacc, *ptry, *pclk;
  if ((s = ws_get(ctx, "march.y", state, &py)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "march.ynew", state, &pyn)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "march.T", state, &pT)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bw.ystage", state, &pys)) != SWF_OK) return s;
  for (int i = 0; i < 7; ++i) {
    char nm[32];
    std::snprintf(nm, sizeof nm, "march.k%d", i);
    if ((s = ws_get(ctx, nm, state, &pk[i])) != SWF_OK) return s;
  }
  const int nbe = (int)std::max<size_t>(1, std::min<size_t>((per_field + 4095) / 4096, 64));
  const int nb = std::max(1, std::min((g.N + 1023) / 1024, (4 * sm_count() + n_inst - 1) / n_inst));
  const size_t nacc = (size_t)3 * nb * n_inst;
  if ((s = ws_get(ctx, "march.ctl", sizeof(StepControl), &pctl)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "march.err_part", sizeof(double) * (size_t)nbe * F, &ppart)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bw.photon", sizeof(double) * 6 * n_inst, &pph)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bw.kph", sizeof(cpx<R>) * n_inst * nt, &pkph)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bw.arows", sizeof(cpx<double>) * 3 * 7 * (size_t)n_inst, &prow)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bw.mpart", sizeof(cpx<double>) * nacc, &pacc)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bw.mtry", sizeof(cpx<double>) * nacc, &ptry)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bw.aclock", sizeof(MarchClock), &pclk)) != SWF_OK) return s;
  cudaError_t e = cudaMemcpyAsync(pph, photon_host, sizeof(double) * 6 * n_inst, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "upload photon table");
  {
    ProfScope ps(ctx, "k_photon_tables", st);
    k_photon_tables<R><<<(n_inst * nt + 127) / 128, 128, 0, st>>>((const double*)pph, g, n_inst, (cpx<R>*)pkph);
  }
  // k_mdot reads its phase row at (clock step + ls) * 7 + stage: a clock at step 0 and a row
  // stride of 7 select the attempt's rows
  MarchClock* clk = (MarchClock*)pclk;
  k_clock_set<<<1, 1, 0, st>>>(clk, t_out, 0.0);
  if ((e = cudaMemsetAsync(py, 0, state, st)) != cudaSuccess) return cuda_status(e, "memset state");
  if ((e = cudaMemsetAsync(pacc, 0, sizeof(cpx<double>) * nacc, st)) != cudaSuccess)
    return cuda_status(e, "memset M accumulators");
  StepControl c0{};
  c0.t = t_out;
  c0.h = (t_in < t_out) ? -std::fabs(h0) : std::fabs(h0);
  if (std::fabs(c0.h) > std::fabs(t_in - t_out)) c0.h = t_in - t_out;
  c0.t_in = t_in;
  c0.span = std::fabs(t_in - t_out);
  c0.rtol = ctx->rtol;
  c0.atol = ctx->atol;
  c0.max_attempts = max_attempts;
  StepControl* ctl = (StepControl*)pctl;
  e = cudaMemcpyAsync(ctl, &c0, sizeof(StepControl), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "upload step control");
  A.y = (cpx<R>*)py;
  A.T = (cpx<R>*)pT;
  {
    StageArgs<R> B = A;  // shapes by timing, before the slots hold anything
    B.nterm = 6;
    for (int q = 0; q < 6; ++q) {
      B.kin[q] = (const cpx<R>*)pk[q + 1];
      B.coef[q] = 0.0;
    }
    B.write_y = 0;
    B.ystage = nullptr;
    B.kout = (cpx<R>*)pk[0];
    B.t = t_out;
    if ((s = autotune_eval<R>(ctx, B, F, st)) != SWF_OK) return s;
  }
  // k_1 = f(t_out, 0)
  A.nterm = 0;
  A.write_y = 0;
  A.kout = (cpx<R>*)pk[0];
  A.t = t_out;
  if ((s = launch_eval<R>(ctx, A, F, st)) != SWF_OK) return s;
  A.ctl = ctl;
  A.ynew = (cpx<R>*)pyn;
  ErrWeights W;
  for (int j = 0; j < 7; ++j) W.db[j] = DP_DB[j];
  const double cell = g.dx[0] * g.dx[1] * g.dx[2];
  auto mdot = [&](const void* ys, int stage) {
    ProfScope ps(ctx, "k_mdot", st);
    k_mdot<R, 1><<<dim3(nb, n_inst), 256, 0, st>>>((const cpx<R>*)ys, A.gcplx, (const cpx<R>*)pkph,
                                                   (const double*)pph, g, (const cpx<double>*)prow, clk, 0, stage,
                                                   7, 1, (cpx<double>*)ptry);
  };
  // the evaluations of an attempt chain through k_last_first (the integrand reads only the stage
  // values); the attempt's last one is closed before the error estimate reads k_7
  const bool chain = !(g.n[1] == 1 && g.n[2] == 1);
  auto attempt = [&]() -> swf_status {
    cudaError_t e1 = cudaMemsetAsync(ptry, 0, sizeof(cpx<double>) * nacc, st);
    if (e1 != cudaSuccess) return cuda_status(e1, "memset attempt sums");
    {
      ProfScope ps(ctx, "k_bw_attempt_rows", st);
      k_bw_attempt_rows<<<n_inst, 32, 0, st>>>(A.fd, (const double*)pph, ctl, cell, (cpx<double>*)prow);
    }
    mdot(py, 0);  // stage 1 of the step: the accepted state
    StageArgs<R> open = A;
    for (int i = 1; i < 7; ++i) {
      int ntm = 0;
      for (int j = 0; j < i; ++j) {
        if (DP_A[i][j] == 0.0) continue;
        A.kin[ntm] = (const cpx<R>*)pk[j];
        A.coef[ntm] = DP_A[i][j];  // times the device-held h in k_first
        ++ntm;
      }
      A.nterm = ntm;
      A.write_y = (i == 6);
      A.kout = (cpx<R>*)pk[i];
      A.c = DP_C[i];
      const bool weighted = i >= 2 && i <= 5;  // b_2 = b_7 = 0
      A.ystage = weighted ? (cpx<R>*)pys : nullptr;
      swf_status r = !chain ? launch_eval<R>(ctx, A, F, st)
                            : (i == 1 ? launch_eval_open<R>(ctx, A, F, st) : launch_eval_chain<R>(ctx, open, A, F, st));
      if (r != SWF_OK) return r;
      open = A;
      if (weighted) mdot(pys, i);
    }
    if (chain) {
      swf_status r = launch_eval_close<R>(ctx, open, F, st);
      if (r != SWF_OK) return r;
    }
    {
      ProfScope ps(ctx, "k_step_error", st);
      k_step_error<R><<<dim3(nbe, F), 256, 0, st>>>(
          (const cpx<R>*)py, (const cpx<R>*)pyn, (const cpx<R>*)pk[0], (const cpx<R>*)pk[1], (const cpx<R>*)pk[2],
          (const cpx<R>*)pk[3], (const cpx<R>*)pk[4], (const cpx<R>*)pk[5], (const cpx<R>*)pk[6], W, ctl, per_field,
          (double*)ppart);
    }
    {
      ProfScope ps(ctx, "k_step_control", st);
      k_step_control<<<1, 32, 0, st>>>(ctl, (const double*)ppart, nbe, F, (double)per_field);
    }
    {
      ProfScope ps(ctx, "k_step_accept", st);
      const size_t n = (size_t)F * per_field;
      k_step_accept<R><<<(unsigned)std::min<size_t>((n + 255) / 256, 4096), 256, 0, st>>>(
          ctl, (cpx<R>*)py, (const cpx<R>*)pyn, (cpx<R>*)pk[0], (const cpx<R>*)pk[6], n);
    }
    {
      ProfScope ps(ctx, "k_mdot_commit", st);
      k_mdot_commit<<<(unsigned)std::min<size_t>((nacc + 255) / 256, 1024), 256, 0, st>>>(
          ctl, (const cpx<double>*)ptry, (cpx<double>*)pacc, nacc);
    }
    return SWF_OK;
  };
  StepControl hc{};
  if ((s = run_attempts(ctx, st, max_attempts, ctl, attempt, &hc)) != SWF_OK) return s;
  ctx->last_accepted = hc.accepted;
  ctx->last_rejected = hc.rejected;
  if (hc.failed) {
    set_error("step-size-controlled march: no convergence (too many attempts or a non-finite error)");
    return SWF_ENUMERIC;
  }
  {
    ProfScope ps(ctx, "k_mdot_final", st);
    k_mdot_final<<<n_inst, 96, 0, st>>>((const cpx<double>*)pacc, nb, (cpx<double>*)macc);
  }
  e = cudaMemcpyAsync(psi_out, py, state, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "copy psi(t_in)");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "Breit-Wheeler march kernels");
  return SWF_OK;
}

swf_status march_bw_adaptive(swf_ctx* ctx, const GridDesc& g, double t_in, double t_out, double h0, int max_attempts,
                             int n_inst, const FieldDesc* fd_host, const double* photon_host, swf_precision prec,
                             void* psi_out, double2* macc, cudaStream_t st) {
  if (prec == SWF_C64)
    return march_bw_adaptive_impl<float>(ctx, g, t_in, t_out, h0, max_attempts, n_inst, fd_host, photon_host,
                                         psi_out, macc, st);
  return march_bw_adaptive_impl<double>(ctx, g, t_in, t_out, h0, max_attempts, n_inst, fd_host, photon_host,
                                        psi_out, macc, st);
}

// ---------------------------------------------------------------- multi-grid march (batching of uneven grids)
// Groups of fields on different grids that share one time grid (t_out, t_in, steps) are marched by
// one launch per pass for all groups: persistent blocks (as many as fit the SMs at once) take work
// items -- one item is one block of one group's pass -- from a device counter, the largest grids'
// items first, and run the single-group kernels' per-block code on them.  A group's lines are
// therefore transformed with exactly the arithmetic of marching that group alone (bitwise the same
// result); the launch only decides which SM does which block, and the whole multi-grid step pair
// is one CUDA graph.  The per-group arguments of every evaluation of the step pair sit in device
// tables, uploaded once before the graph is captured (the slots rotate with period two).

constexpr int kMaxMultiGroups = 8;
constexpr int kMultiCounters = 128;  // work counters of one step pair (one per grouped launch)

struct MultiPlan {
  int items;                       // work items of the launch
  int first[kMaxMultiGroups + 1];  // first item of queue position q (largest grids first)
  int gid[kMaxMultiGroups];        // table index of the group at queue position q
  int gx[kMaxMultiGroups];         // blocks per field of that group in this pass
  int shape[kMaxMultiGroups];      // rows per block (x passes) or log2 of the tile width (y, z passes)
  int ld[kMaxMultiGroups];         // padded line stride
};

// Breit-Wheeler integrand arguments of one group (one photon per instance).
template <typename R>
struct MdotArgs {
  const cpx<R>* ys;
  const cpx<R>* gcplx;
  const cpx<R>* kph;
  const double* photon;
  const cpx<double>* ptab;
  cpx<double>* acc;
  GridDesc g;
  int tab_stride;
  int nb;  // blocks per instance (the split of the single-group march)
};

// Persistent loop over the work items of a grouped launch: body(args, bx, by, shape, ld) with the
// item's group arguments copied into shared memory.
template <typename Args, typename Body>
__device__ __forceinline__ void multi_loop(const Args* __restrict__ tab, const MultiPlan& P, int* counter,
                                           Body&& body) {
  __shared__ __align__(16) Args sA;
  __shared__ MultiPlan sP;
  __shared__ int s_item;
  if (threadIdx.x == 0) sP = P;
  int cur = -1;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = s_item;
    if (item >= sP.items) break;
    int q = 0;
    while (q + 1 < kMaxMultiGroups && item >= sP.first[q + 1]) ++q;
    if (q != cur) {
      const int* src = reinterpret_cast<const int*>(tab + sP.gid[q]);
      int* dst = reinterpret_cast<int*>(&sA);
      for (int i = threadIdx.x; i < (int)(sizeof(Args) / sizeof(int)); i += blockDim.x) dst[i] = __ldg(src + i);
      __syncthreads();
      cur = q;
    }
    const int local = item - sP.first[q];
    body(sA, local % sP.gx[q], local / sP.gx[q], sP.shape[q], sP.ld[q]);
    __syncthreads();  // shared memory and s_item are reused by the next item
  }
}

// The per-group arguments come from shared memory instead of the constant bank, which costs the
// kernels registers; the bounds keep them at the occupancy of the single-group kernels (a few
// bytes of spills in complex64, about a hundred in complex128).
template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 2) k_first_multi(const StageArgs<R>* __restrict__ tab, MultiPlan P, int only_x,
                                                     int* counter) {
  multi_loop(tab, P, counter, [&](const StageArgs<R>& A, int bx, int f, int rows, int ld) {
    first_body<R>(A, bx, f, rows, ld, only_x);
  });
}

template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 2) k_mid_multi(const StageArgs<R>* __restrict__ tab, MultiPlan P, int axis,
                                                   int do_fwd, int do_h0, int do_inv, int* counter) {
  multi_loop(tab, P, counter, [&](const StageArgs<R>& A, int bx, int f, int lgtx, int ld) {
    mid_body<R>(A, bx, f, axis, lgtx, ld, do_fwd, do_h0, do_inv);
  });
}

template <typename R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 3 : 2) k_last_multi(const StageArgs<R>* __restrict__ tab, MultiPlan P, int* counter) {
  multi_loop(tab, P, counter, [&](const StageArgs<R>& A, int bx, int f, int rows, int ld) {
    last_body<R>(A, bx, f, rows, ld);
  });
}

template <typename R>
__global__ void __launch_bounds__(256) k_mdot_multi(const MdotArgs<R>* __restrict__ tab, MultiPlan P,
                                                    const MarchClock* clk, int ls, int stage, int* counter) {
  multi_loop(tab, P, counter, [&](const MdotArgs<R>& M, int bx, int by, int, int) {
    mdot_body<R, 1>(M.ys, M.gcplx, M.kph, M.photon, M.g, M.ptab, clk, ls, stage, M.tab_stride, 1, M.acc, bx, by,
                    M.nb);
  });
}

template <typename R>
static swf_status set_multi_attrs() {
  static std::atomic<bool> done[64];
  const int dv = dev_slot();
  if (done[dv].load(std::memory_order_acquire)) return SWF_OK;
  cudaError_t e;
  e = cudaFuncSetAttribute(k_first_multi<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmemTune);
  if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(k_first_multi)");
  e = cudaFuncSetAttribute(k_mid_multi<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmemTune);
  if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(k_mid_multi)");
  e = cudaFuncSetAttribute(k_last_multi<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPassSmemTune);
  if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(k_last_multi)");
  done[dv].store(true, std::memory_order_release);
  return SWF_OK;
}

// Blocks of a persistent grouped launch: as many as can be resident at once (at most one per item).
template <typename K>
static int persistent_blocks(K kernel, size_t smem, int items, int threads = kThreads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  return std::max(1, std::min(items, per_sm * sm_count()));
}

// Queue positions of the groups: largest grids first (their items take longest).
static std::vector<int> multi_order(const std::vector<MultiGroup>& G) {
  std::vector<int> ord(G.size());
  for (size_t i = 0; i < G.size(); ++i) ord[i] = (int)i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return G[a].g.N > G[b].g.N; });
  return ord;
}

static MultiPlan make_plan(const std::vector<int>& ord, const std::vector<int>& gx, const std::vector<int>& per,
                           const std::vector<int>& shape, const std::vector<int>& ld) {
  MultiPlan P;
  std::memset(&P, 0, sizeof(P));
  int acc = 0;
  for (int q = 0; q < kMaxMultiGroups; ++q) {
    P.first[q] = acc;
    if (q < (int)ord.size()) {
      const int gi = ord[q];
      P.gid[q] = gi;
      P.gx[q] = gx[gi];
      P.shape[q] = shape[gi];
      P.ld[q] = ld[gi];
      acc += gx[gi] * per[gi];
    }
  }
  P.first[kMaxMultiGroups] = acc;
  P.items = acc;
  return P;
}

template <typename R>
static swf_status march_multi_impl(swf_ctx* ctx, const std::vector<MultiGroup>& G, double t_in, double t_out,
                                   int n_steps, int bw, cudaStream_t st) {
  const int ng = (int)G.size();
  constexpr int esz = (int)sizeof(cpx<R>);
  swf_status s = set_multi_attrs<R>();
  if (s != SWF_OK) return s;
  const int ny0 = G[0].g.n[1], nz0 = G[0].g.n[2];
  const bool only_x = (ny0 == 1 && nz0 == 1);
  std::vector<StageArgs<R>> base(ng);
  std::vector<void*> pk(7 * (size_t)ng), pys(ng, nullptr), ppart(ng, nullptr);
  std::vector<MdotArgs<R>> mdot(ng);
  std::vector<int> nb(ng, 1);
  const double h = (t_in - t_out) / n_steps;
  cudaError_t e;
  for (int gi = 0; gi < ng; ++gi) {
    const MultiGroup& M = G[gi];
    const GridDesc& g = M.g;
    const int F = M.F;
    const std::string tag = "mg" + std::to_string(gi);
    if ((s = prepare_args<R>(ctx, g, F, M.fd, &base[gi], tag.c_str(), st)) != SWF_OK) return s;
    const size_t state = (size_t)F * 4 * g.N * esz;
    void *py = nullptr, *pT = nullptr;
    if ((s = ws_get(ctx, tag + ".y", state, &py)) != SWF_OK) return s;
    if ((s = ws_get(ctx, tag + ".T", state, &pT)) != SWF_OK) return s;
    for (int i = 0; i < 7; ++i)
      if ((s = ws_get(ctx, tag + ".k" + std::to_string(i), state, &pk[7 * gi + i])) != SWF_OK) return s;
    if ((e = cudaMemsetAsync(py, 0, state, st)) != cudaSuccess) return cuda_status(e, "memset state");
    base[gi].y = (cpx<R>*)py;
    base[gi].T = (cpx<R>*)pT;
    if ((s = state_low_part<R>(ctx, tag + ".ylo", state, &base[gi], st)) != SWF_OK) return s;
    if (bw) {
      const int n_inst = F / 2;
      const int nt = g.n[0] + g.n[1] + g.n[2];
      void *pph = nullptr, *pkph = nullptr, *ptab = nullptr;
      if ((s = ws_get(ctx, tag + ".ystage", state, &pys[gi])) != SWF_OK) return s;
      if ((s = ws_get(ctx, tag + ".photon", sizeof(double) * 6 * n_inst, &pph)) != SWF_OK) return s;
      if ((s = ws_get(ctx, tag + ".kph", sizeof(cpx<R>) * n_inst * nt, &pkph)) != SWF_OK) return s;
      // the same split of the integrand sums as the single-group march of this group
      nb[gi] = std::max(1, std::min((g.N + 1023) / 1024, (4 * sm_count() + n_inst - 1) / n_inst));
      if ((s = ws_get(ctx, tag + ".ptab", sizeof(cpx<double>) * 3 * 7 * (size_t)n_steps * n_inst, &ptab)) != SWF_OK)
        return s;
      if ((s = ws_get(ctx, tag + ".mpart", sizeof(cpx<double>) * 3 * (size_t)nb[gi] * n_inst, &ppart[gi])) != SWF_OK)
        return s;
      if ((e = cudaMemcpyAsync(pph, M.photon, sizeof(double) * 6 * n_inst, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_status(e, "upload photon table");
      {
        ProfScope ps(ctx, "k_photon_tables", st);
        k_photon_tables<R><<<(n_inst * nt + 127) / 128, 128, 0, st>>>((const double*)pph, g, n_inst, (cpx<R>*)pkph);
      }
      {
        const long total = (long)n_inst * n_steps * 7;
        ProfScope ps(ctx, "k_bw_phase_table", st);
        k_bw_phase_table<<<(int)std::min((total + 127) / 128, 4096L), 128, 0, st>>>(
            base[gi].fd, (const double*)pph, n_inst, 1, n_steps, t_out, h, g.dx[0] * g.dx[1] * g.dx[2], 1,
            (cpx<double>*)ptab);
      }
      if ((e = cudaMemsetAsync(ppart[gi], 0, sizeof(cpx<double>) * 3 * (size_t)nb[gi] * n_inst, st)) != cudaSuccess)
        return cuda_status(e, "memset M accumulators");
      mdot[gi] = MdotArgs<R>{(const cpx<R>*)pys[gi], base[gi].gcplx, (const cpx<R>*)pkph, (const double*)pph,
                             (const cpx<double>*)ptab, (cpx<double>*)ppart[gi], g, 7 * n_steps, nb[gi]};
    }
    {  // launch shapes of this group by timing (as for a single-group march)
      StageArgs<R> B = base[gi];
      B.nterm = 6;
      for (int q = 0; q < 6; ++q) {
        B.kin[q] = (const cpx<R>*)pk[7 * gi + q + 1];
        B.coef[q] = 0.0;
      }
      B.write_y = 0;
      B.ystage = nullptr;
      B.kout = (cpx<R>*)pk[7 * gi];
      B.t = t_out;
      if ((s = autotune_eval<R>(ctx, B, F, st)) != SWF_OK) return s;
    }
  }
  // Per-pass plans.  The lead group (the largest grid, first in the queue) keeps its tuned shape
  // and thread count; it fixes the launch's shared memory per block, and every other group takes
  // the largest shape that fits that budget (more rows, or wider tiles, for smaller grids), so that
  // its blocks do not reserve shared memory they leave unused.
  const std::vector<int> ord = multi_order(G);
  const int lead = ord[0];
  std::vector<int> fper(ng), xg(ng), xrows(ng), xld(ng);
  int xthr = kThreads;
  size_t xsmem = 0;
  {
    const GridDesc& g = G[lead].g;
    const int nrows = g.n[1] * g.n[2];
    const int xv = tune_lookup(ctx, tune_key('x', esz, g.n[0], nrows, 0, G[lead].F),
                               4 * x_rows<R>(g.n[0], nrows, G[lead].F));
    xthr = (xv & 3) ? kThreads / 2 : kThreads;
    xsmem = (size_t)2 * 4 * std::max(1, xv >> 2) * padded_len(g.n[0]) * esz;
  }
  for (int gi = 0; gi < ng; ++gi) {
    const GridDesc& g = G[gi].g;
    fper[gi] = G[gi].F;
    const int nrows = g.n[1] * g.n[2];
    xld[gi] = padded_len(g.n[0]);
    const size_t line = (size_t)2 * 4 * xld[gi] * esz;
    xrows[gi] = (int)std::max<size_t>(1, std::min<size_t>(std::min<size_t>(xsmem / line, 64), nrows));
    xg[gi] = (nrows + xrows[gi] - 1) / xrows[gi];
    xsmem = std::max(xsmem, (size_t)xrows[gi] * line);
  }
  const MultiPlan px = make_plan(ord, xg, fper, xrows, xld);
  struct MidPass { int axis, fwd, h0, inv; MultiPlan plan; size_t smem; int blocks, threads; };
  std::vector<MidPass> mids;
  if (!only_x) {
    std::vector<std::array<int, 4>> combos;
    if (ny0 > 1 && nz0 > 1) combos = {{1, 1, 0, 0}, {2, 1, 1, 1}, {1, 0, 0, 1}};
    else combos = {{ny0 > 1 ? 1 : 2, 1, 1, 1}};
    for (const auto& cb : combos) {
      const int axis = cb[0];
      auto tuned = [&](int gi) {
        const GridDesc& g = G[gi].g;
        const int other = axis == 1 ? g.n[2] : g.n[1];
        const int lg_h = mid_shape<R>(g.n[axis], g.n[0], (long)other * G[gi].F).lgtx;
        return tune_lookup(ctx, tune_key('m', esz, axis * 8 + cb[1] * 4 + cb[2] * 2 + cb[3], g.n[axis], g.n[0],
                                         (long)other * G[gi].F), 4 * lg_h);
      };
      const int mv_lead = tuned(lead);
      const size_t budget = mid_shape_lg<R>(G[lead].g.n[axis], mv_lead >> 2).smem;
      std::vector<int> mg(ng), lg(ng), ld(ng);
      size_t sm = 0;
      for (int gi = 0; gi < ng; ++gi) {
        const GridDesc& g = G[gi].g;
        const int other = axis == 1 ? g.n[2] : g.n[1];
        int l = gi == lead ? (mv_lead >> 2) : mid_max_lg<R>(g.n[axis], g.n[0], budget);
        const MidShape ms = mid_shape_lg<R>(g.n[axis], l);
        lg[gi] = ms.lgtx;
        ld[gi] = ms.ld;
        mg[gi] = ((g.n[0] + (1 << ms.lgtx) - 1) >> ms.lgtx) * other;
        sm = std::max(sm, ms.smem);
      }
      MidPass mp{axis, cb[1], cb[2], cb[3], make_plan(ord, mg, fper, lg, ld), sm, 0,
                 (mv_lead & 3) ? kThreads / 2 : kThreads};
      mp.blocks = persistent_blocks(k_mid_multi<R>, sm, mp.plan.items, mp.threads);
      mids.push_back(mp);
    }
  }
  const int xfb = persistent_blocks(k_first_multi<R>, xsmem, px.items, xthr);
  const int xlb = persistent_blocks(k_last_multi<R>, xsmem, px.items, xthr);
  MultiPlan pd;
  int dblocks = 0;
  if (bw) {
    std::vector<int> ones(ng, 1), zero(ng, 0), ninst(ng);
    for (int gi = 0; gi < ng; ++gi) ninst[gi] = G[gi].F / 2;
    pd = make_plan(ord, nb, ninst, zero, zero);
    dblocks = persistent_blocks(k_mdot_multi<R>, 0, pd.items);
  }
  // argument tables of every evaluation of a step pair: entry 0 the first evaluation k_1 = f(t_out, 0),
  // then (ls, stage) for ls = 0, 1 and stages 1..6, with the slot rotation of the single-group march
  const int n_ev = 1 + 12;
  std::vector<StageArgs<R>> tab((size_t)n_ev * ng);
  std::vector<std::array<int, 7>> slot(ng);
  for (int gi = 0; gi < ng; ++gi) {
    for (int i = 0; i < 7; ++i) slot[gi][i] = i;
    StageArgs<R> A = base[gi];
    A.nterm = 0;
    A.write_y = 0;
    A.kout = (cpx<R>*)pk[7 * gi + slot[gi][0]];
    A.ls = 0;
    A.c = 0.0;
    A.ystage = nullptr;
    A.t = t_out;
    tab[gi] = A;
  }
  void* pclk = nullptr;
  if ((s = ws_get(ctx, "mg.clock", sizeof(MarchClock), &pclk)) != SWF_OK) return s;
  MarchClock* clk = (MarchClock*)pclk;
  for (int ls = 0; ls < 2; ++ls) {
    for (int i = 1; i < 7; ++i) {
      for (int gi = 0; gi < ng; ++gi) {
        StageArgs<R> A = base[gi];
        int nt = 0;
        for (int j = 0; j < i; ++j) {
          if (DP_A[i][j] == 0.0) continue;
          A.kin[nt] = (const cpx<R>*)pk[7 * gi + slot[gi][j]];
          A.coef[nt] = h * DP_A[i][j];
          ++nt;
        }
        A.nterm = nt;
        A.write_y = (i == 6);
        A.kout = (cpx<R>*)pk[7 * gi + slot[gi][i]];
        A.ls = ls;
        A.c = DP_C[i];
        A.clk = clk;
        A.ystage = (bw && i >= 2) ? (cpx<R>*)pys[gi] : nullptr;
        tab[(size_t)(1 + 6 * ls + (i - 1)) * ng + gi] = A;
      }
    }
    for (int gi = 0; gi < ng; ++gi) std::swap(slot[gi][0], slot[gi][6]);
  }
  void *ptabs = nullptr, *pmd = nullptr, *pcnt = nullptr;
  if ((s = ws_get(ctx, "mg.tables", sizeof(StageArgs<R>) * tab.size(), &ptabs)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "mg.counters", sizeof(int) * kMultiCounters, &pcnt)) != SWF_OK) return s;
  if ((e = cudaMemcpyAsync(ptabs, tab.data(), sizeof(StageArgs<R>) * tab.size(), cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return cuda_status(e, "upload multi-grid tables");
  if (bw) {
    if ((s = ws_get(ctx, "mg.mdot", sizeof(MdotArgs<R>) * ng, &pmd)) != SWF_OK) return s;
    if ((e = cudaMemcpyAsync(pmd, mdot.data(), sizeof(MdotArgs<R>) * ng, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return cuda_status(e, "upload multi-grid integrand table");
  }
  const StageArgs<R>* dtab = (const StageArgs<R>*)ptabs;
  int* cnt = (int*)pcnt;
  int ci = 0;  // next counter of the recorded sequence
  auto eval = [&](int ev) {
    const StageArgs<R>* t = dtab + (size_t)ev * ng;
    {
      ProfScope ps(ctx, "k_first_multi", st);
      k_first_multi<R><<<xfb, xthr, xsmem, st>>>(t, px, only_x ? 1 : 0, cnt + ci++);
    }
    if (only_x) return;
    for (const MidPass& mp : mids) {
      ProfScope ps(ctx, "k_mid_multi", st);
      k_mid_multi<R><<<mp.blocks, mp.threads, mp.smem, st>>>(t, mp.plan, mp.axis, mp.fwd, mp.h0, mp.inv, cnt + ci++);
    }
    ProfScope ps(ctx, "k_last_multi", st);
    k_last_multi<R><<<xlb, xthr, xsmem, st>>>(t, px, cnt + ci++);
  };
  auto step = [&](int ls) {
    for (int i = 1; i < 7; ++i) {
      eval(1 + 6 * ls + (i - 1));
      if (bw && i >= 2) {
        ProfScope ps(ctx, "k_mdot_multi", st);
        k_mdot_multi<R><<<dblocks, kThreads, 0, st>>>((const MdotArgs<R>*)pmd, pd, clk, ls, i, cnt + ci++);
      }
    }
  };
  // work counters used per step pair: every stage's passes, and the integrand at stages 2..6
  const int per_eval = only_x ? 1 : 2 + (int)mids.size();
  const int per_pair = 2 * (6 * per_eval + (bw ? 5 : 0));
  if (per_pair > kMultiCounters) {
    set_error("multi-grid march: too many launches per step pair");
    return SWF_EUNSUPPORTED;
  }
  k_clock_set<<<1, 1, 0, st>>>(clk, t_out, h);
  if ((e = cudaMemsetAsync(cnt, 0, sizeof(int) * kMultiCounters, st)) != cudaSuccess) return cuda_status(e, "reset work queues");
  ci = 0;
  eval(0);  // k_1 = f(t_out, 0) (the integrand of Eq. 17 vanishes at psi_s(t_out) = 0)
  auto pair = [&]() -> swf_status {
    cudaError_t r = cudaMemsetAsync(cnt, 0, sizeof(int) * kMultiCounters, st);
    if (r != cudaSuccess) return cuda_status(r, "reset work queues");
    ci = 0;
    step(0);
    step(1);
    return SWF_OK;
  };
  if ((s = run_step_pairs(ctx, st, n_steps / 2, clk, pair)) != SWF_OK) return s;
  if (n_steps % 2) {
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int) * kMultiCounters, st)) != cudaSuccess) return cuda_status(e, "reset work queues");
    ci = 0;
    step(0);
  }
  for (int gi = 0; gi < ng; ++gi) {
    const size_t state = (size_t)G[gi].F * 4 * G[gi].g.N * esz;
    if (bw) {
      ProfScope ps(ctx, "k_mdot_final", st);
      k_mdot_final<<<G[gi].F / 2, 96, 0, st>>>((const cpx<double>*)ppart[gi], nb[gi], (cpx<double>*)G[gi].macc);
    }
    if ((e = cudaMemcpyAsync(G[gi].psi_out, base[gi].y, state, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return cuda_status(e, "copy psi(t_in)");
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_status(e, "multi-grid march kernels");
  // the host tables above are the sources of asynchronous uploads
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(e, "multi-grid march");
  ctx->multi_marches += 1;
  return SWF_OK;
}

bool multi_compatible(const GridDesc& a, const GridDesc& b) {
  return (a.n[1] > 1) == (b.n[1] > 1) && (a.n[2] > 1) == (b.n[2] > 1);
}

swf_status march_multi(swf_ctx* ctx, const std::vector<MultiGroup>& groups, double t_in, double t_out, int n_steps,
                       swf_precision prec, int bw, cudaStream_t st) {
  if (groups.empty() || (int)groups.size() > kMaxMultiGroups) {
    set_error("multi-grid march: 1 to 8 groups");
    return SWF_EINVAL;
  }
  for (const MultiGroup& M : groups) {
    if (!multi_compatible(M.g, groups[0].g) || M.F < 1 || (bw && (M.F % 2 || !M.photon || !M.macc))) {
      set_error("multi-grid march: groups must share the non-trivial axes (and carry U, V pairs and photons)");
      return SWF_EINVAL;
    }
  }
  if (prec == SWF_C64) return march_multi_impl<float>(ctx, groups, t_in, t_out, n_steps, bw, st);
  return march_multi_impl<double>(ctx, groups, t_in, t_out, n_steps, bw, st);
}

// Plain marches of several groups (the spin reuse of march_fields within each group).
swf_status march_fields_multi(swf_ctx* ctx, const std::vector<MultiGroup>& groups, double t_in, double t_out,
                              int n_steps, swf_precision prec, cudaStream_t st) {
  const int ng = (int)groups.size();
  std::vector<MultiGroup> todo(groups);
  std::vector<std::vector<int>> rep(ng), sgn(ng);
  std::vector<std::vector<FieldDesc>> uniq(ng);
  const size_t elem = prec == SWF_C64 ? 8 : 16;
  swf_status s;
  for (int gi = 0; gi < ng; ++gi) {
    const MultiGroup& M = groups[gi];
    const int n_u = ctx->dedupe ? dedupe_fields(M.g, M.F, M.fd, rep[gi], sgn[gi], uniq[gi]) : M.F;
    ctx->fields_marched += n_u;
    if (n_u == M.F) {
      rep[gi].clear();
      continue;
    }
    void* pu = nullptr;
    if ((s = ws_get(ctx, "mg.unique" + std::to_string(gi), (size_t)n_u * 4 * M.g.N * elem, &pu)) != SWF_OK) return s;
    todo[gi].F = n_u;
    todo[gi].fd = uniq[gi].data();
    todo[gi].psi_out = pu;
  }
  if ((s = march_multi(ctx, todo, t_in, t_out, n_steps, prec, 0, st)) != SWF_OK) return s;
  for (int gi = 0; gi < ng; ++gi) {
    if (rep[gi].empty()) continue;
    const MultiGroup& M = groups[gi];
    void* ptab = nullptr;
    if ((s = ws_get(ctx, "mg.unique_map" + std::to_string(gi), sizeof(int) * 2 * (size_t)M.F, &ptab)) != SWF_OK)
      return s;
    std::vector<int> tabv(rep[gi]);
    tabv.insert(tabv.end(), sgn[gi].begin(), sgn[gi].end());
    cudaError_t e = cudaMemcpyAsync(ptab, tabv.data(), sizeof(int) * 2 * (size_t)M.F, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_status(e, "upload field map");
    const dim3 grid((unsigned)std::min<size_t>((M.g.N + 255) / 256, 1024), M.F, 4);
    ProfScope ps(ctx, "k_expand_fields", st);
    if (prec == SWF_C64)
      k_expand_fields<float><<<grid, 256, 0, st>>>((const cpx<float>*)todo[gi].psi_out, (const int*)ptab,
                                                   (const int*)ptab + M.F, (size_t)M.g.N, (cpx<float>*)M.psi_out);
    else
      k_expand_fields<double><<<grid, 256, 0, st>>>((const cpx<double>*)todo[gi].psi_out, (const int*)ptab,
                                                    (const int*)ptab + M.F, (size_t)M.g.N, (cpx<double>*)M.psi_out);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, "expand fields");
    e = cudaStreamSynchronize(st);  // the host table must outlive its upload
    if (e != cudaSuccess) return cuda_status(e, "expand fields");
  }
  return SWF_OK;
}

}  // namespace swf
