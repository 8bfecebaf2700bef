// Full pair numbers N(m, n) of Eq. 8 for every electron m of one list and positron n of another,
// all in one field, grid and time window (Sec. II, Eqs. 8-9; Sec. II.A: scans over momenta).
//
// Instead of one U and one V march per pair, every electron is marched once (U waves) and every
// positron once (V waves), and the four overlaps of Eq. 8 become complex matrix products over
// the grid (K = 4 N: components x sites), in FP64:
//   C(m, n) = dx^d sum_x U_m^+(x) V_back,n(x)              (position space)
//   A(m, n) = dx^d sum_x U_back,m^+(x) V_n(x)              (position space)
//   B(m, n) = L^-d sum_j (P_+(k_j) U~_m(j))^+ V~_n(j)      (grid modes, P_+- energy projectors)
//   D(m, n) = L^-d sum_j (P_-(k_j) U~_m(j))^+ V~_n(j)
// with U~, V~ the continuum-normalised transforms and the backgrounds U_back = u_s(p)
// e^{-i(p0 t - p.x)}, V_back = v_r(q) e^{i(q0 t - q.x)} at t = t_in.  The sums over s' and the
// grid modes Q of Eq. 8 are the projectors (sum_s' u u^+ = P_+, sum_s' v v^+ = P_-), as in the
// single-pair path.  N = |C + D|^2 = |A + B|^2.
#include <algorithm>
#include <cstring>
#include <vector>

#include "swf_internal.h"

namespace swf {
namespace pairs {

constexpr int TM = 32, TN = 32, TK = 16;  // output tile and k step of the product kernel

// part[s][m][n] = sum over k in split s of conj(X[m][k]) Y[n][k]; X: M rows, Y: Nn rows, both
// K long and contiguous.  256 threads, 2 x 2 outputs each; the splits are added in order by
// k_sum_splits (deterministic).
__global__ void __launch_bounds__(256) k_gemm_cn(const cpx<double>* __restrict__ X, const cpx<double>* __restrict__ Y,
                                                 int M, int Nn, long K, long kchunk, cpx<double>* part) {
  __shared__ cpx<double> xs[TK][TM + 1];
  __shared__ cpx<double> ys[TK][TN + 1];
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  const long k0 = blockIdx.z * kchunk;
  const long k1 = std::min(K, k0 + kchunk);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  cpx<double> acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = mk<double>(0, 0);
  for (long kb = k0; kb < k1; kb += TK) {
    // tiles: TM x TK of X and TN x TK of Y (k fastest in memory: coalesced along k)
    for (int e = threadIdx.x; e < TM * TK; e += blockDim.x) {
      const int r = e / TK, c = e % TK;
      const long k = kb + c;
      xs[c][r] = (m0 + r < M && k < k1) ? X[(size_t)(m0 + r) * K + k] : mk<double>(0, 0);
      ys[c][r] = (n0 + r < Nn && k < k1) ? Y[(size_t)(n0 + r) * K + k] : mk<double>(0, 0);
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < TK; ++c) {
      const cpx<double> x0 = xs[c][ty], x1 = xs[c][ty + 16];
      const cpx<double> y0 = ys[c][tx], y1 = ys[c][tx + 16];
      acc[0][0] = acc[0][0] + cdot(x0, y0);
      acc[0][1] = acc[0][1] + cdot(x0, y1);
      acc[1][0] = acc[1][0] + cdot(x1, y0);
      acc[1][1] = acc[1][1] + cdot(x1, y1);
    }
    __syncthreads();
  }
  cpx<double>* out = part + (size_t)blockIdx.z * M * Nn;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < M && n < Nn) out[(size_t)m * Nn + n] = acc[i][j];
    }
}

// out[m][n] = scale sum_s part[s][m][n], splits in order.
__global__ void k_sum_splits(const cpx<double>* __restrict__ part, int S, long MN, double scale, cpx<double>* out) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < MN; i += (long)gridDim.x * blockDim.x) {
    cpx<double> s = mk<double>(0, 0);
    for (int k = 0; k < S; ++k) s = s + part[(size_t)k * MN + i];
    out[i] = scale * s;
  }
}

template <typename R>
__global__ void k_widen(const cpx<R>* __restrict__ in, cpx<double>* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = cvt<double>(in[i]);
}

// Background plane waves on the grid at t_in: w[8] = spinor (re, im) x 4, mom = momentum of the
// exponent e^{i sgn (mom.x - E t)} (U: sgn = +1, mom = p; V: sgn = -1, mom = q).  Trivial axes
// carry no phase (their momentum is the marched wave's own, the same on both sides).
struct Wave {
  double w[8];
  double mom[3];
  double sgn;
};

__global__ void k_plane_waves(const Wave* wv, GridDesc g, double t, cpx<double>* out) {
  const int f = blockIdx.y;
  const Wave W = wv[f];
  const double E = sqrt(1.0 + W.mom[0] * W.mom[0] + W.mom[1] * W.mom[1] + W.mom[2] * W.mom[2]);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < g.N; j += gridDim.x * blockDim.x) {
    const int ix = j % g.n[0];
    const int iy = (j / g.n[0]) % g.n[1];
    const int iz = j / (g.n[0] * g.n[1]);
    const int id[3] = {ix, iy, iz};
    double ph = -E * t;
    for (int a = 0; a < 3; ++a)
      if (g.n[a] > 1) ph += W.mom[a] * (g.x0[a] + id[a] * g.dx[a]);
    double sn, cs;
    sincos(W.sgn * ph, &sn, &cs);
    const cpx<double> e = mk<double>(cs, sn);
#pragma unroll
    for (int a = 0; a < 4; ++a)
      out[((size_t)f * 4 + a) * g.N + j] = e * mk<double>(W.w[2 * a], W.w[2 * a + 1]);
  }
}

// out[sgn][m] = P_sgn(kappa_j) spec[m] per grid mode (P_+- = (1 +- H0/E)/2), sgn = + first.
__global__ void k_project(const cpx<double>* __restrict__ spec, GridDesc g, const double* __restrict__ Ku, int n_f,
                          cpx<double>* __restrict__ out) {
  const int f = blockIdx.y;
  const cpx<double>* u = spec + (size_t)f * 4 * g.N;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < g.N; j += gridDim.x * blockDim.x) {
    const int ix = j % g.n[0];
    const int iy = (j / g.n[0]) % g.n[1];
    const int iz = j / (g.n[0] * g.n[1]);
    const double kx = g.n[0] > 1 ? mode_kappa(ix, g.n[0], g.L[0]) : Ku[0];
    const double ky = g.n[1] > 1 ? mode_kappa(iy, g.n[1], g.L[1]) : Ku[1];
    const double kz = g.n[2] > 1 ? mode_kappa(iz, g.n[2], g.L[2]) : Ku[2];
    const double iE = 1.0 / sqrt(1.0 + kx * kx + ky * ky + kz * kz);
    cpx<double> a[4], h[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) a[c] = u[(size_t)c * g.N + j];
    // H0(kappa) a = (alpha.kappa + beta) a, Dirac representation
    h[0] = a[0] + kz * a[2] + kx * a[3] + ky * mul_mi(a[3]);
    h[1] = a[1] + kx * a[2] + ky * mul_i(a[2]) - kz * a[3];
    h[2] = kz * a[0] + kx * a[1] + ky * mul_mi(a[1]) - a[2];
    h[3] = kx * a[0] + ky * mul_i(a[0]) - kz * a[1] - a[3];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      out[((size_t)f * 4 + c) * g.N + j] = 0.5 * (a[c] + iE * h[c]);
      out[((size_t)(n_f + f) * 4 + c) * g.N + j] = 0.5 * (a[c] - iE * h[c]);
    }
  }
}

// results[m][n] from the four overlap matrices (B and D stacked: rows m and n_e + m).
__global__ void k_pair_results(const cpx<double>* __restrict__ Cm, const cpx<double>* __restrict__ Am,
                               const cpx<double>* __restrict__ BDm, const double* normU, const double* normV, int n_e,
                               int n_p, swf_result* res) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_e * n_p; i += gridDim.x * blockDim.x) {
    const int m = i / n_p, n = i % n_p;
    const cpx<double> C = Cm[i], A = Am[i], B = BDm[(size_t)m * n_p + n], D = BDm[(size_t)(n_e + m) * n_p + n];
    swf_result o;
    o.amp[0] = C.x; o.amp[1] = C.y;
    o.amp[2] = D.x; o.amp[3] = D.y;
    o.amp[4] = A.x; o.amp[5] = A.y;
    o.amp[6] = B.x; o.amp[7] = B.y;
    const cpx<double> CD = C + D, AB = A + B;
    o.prob[0] = CD.x * CD.x + CD.y * CD.y;
    o.prob[1] = AB.x * AB.x + AB.y * AB.y;
    o.diag[0] = normU[m];
    o.diag[1] = normV[n];
    res[i] = o;
  }
}

int sms() {
  int dev = 0, n = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    n = 152;
  return n;
}

// out = scale X^+ Y (M x Nn) with split K, through the part buffer.
swf_status gemm_cn(swf_ctx* ctx, const cpx<double>* X, const cpx<double>* Y, int M, int Nn, long K, double scale,
                   cpx<double>* out, const char* tag, cudaStream_t st) {
  const int tiles = ((Nn + TN - 1) / TN) * ((M + TM - 1) / TM);
  long S = std::max(1L, (2L * sms() + tiles - 1) / tiles);
  S = std::min(S, std::max(1L, K / 256));
  S = std::min(S, 1024L);
  long kchunk = (K + S - 1) / S;
  kchunk = (kchunk + TK - 1) / TK * TK;
  S = (K + kchunk - 1) / kchunk;
  void* part = nullptr;
  swf_status s = ws_get(ctx, "pairs.part", sizeof(cpx<double>) * (size_t)S * M * Nn, &part);
  if (s != SWF_OK) return s;
  {
    ProfScope ps(ctx, "k_gemm_cn", st);
    k_gemm_cn<<<dim3((Nn + TN - 1) / TN, (M + TM - 1) / TM, (unsigned)S), 256, 0, st>>>(X, Y, M, Nn, K, kchunk,
                                                                                        (cpx<double>*)part);
  }
  {
    ProfScope ps(ctx, "k_sum_splits", st);
    const long MN = (long)M * Nn;
    k_sum_splits<<<(int)std::min((MN + 255) / 256, 4096L), 256, 0, st>>>((const cpx<double>*)part, (int)S, MN, scale,
                                                                          out);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, tag);
  return SWF_OK;
}

bool same_grid(const swf_grid& a, const swf_grid& b) {
  for (int k = 0; k < 3; ++k) {
    if (a.n[k] != b.n[k]) return false;
    if (a.n[k] > 1 && a.L[k] != b.L[k]) return false;
  }
  return a.t_in == b.t_in && a.t_out == b.t_out && a.n_steps == b.n_steps;
}

bool same_field(const swf_field& a, const swf_field& b) {
  if (a.kind != b.kind) return false;
  for (int k = 0; k < 8; ++k)
    if (a.prm[k] != b.prm[k]) return false;
  return true;
}

}  // namespace pairs
}  // namespace swf

using namespace swf;

extern "C" swf_status swf_pair_matrix(swf_ctx* ctx, int n_e, const swf_instance* electrons, int n_p,
                                      const swf_instance* positrons, swf_precision prec, swf_result* results) {
  if (!ctx) { set_error("ctx is NULL"); return SWF_EINVAL; }
  if (n_e < 1 || n_p < 1 || !electrons || !positrons || !results) {
    set_error("swf_pair_matrix: need n_e >= 1, n_p >= 1 and non-NULL arrays");
    return SWF_EINVAL;
  }
  swf_status s = validate_instances(n_e, electrons, prec);
  if (s != SWF_OK) return s;
  if ((s = validate_instances(n_p, positrons, prec)) != SWF_OK) return s;
  const swf_instance& i0 = electrons[0];
  for (int k = 0; k < n_e + n_p; ++k) {
    const swf_instance& in = k < n_e ? electrons[k] : positrons[k - n_e];
    if (!pairs::same_grid(in.grid, i0.grid) || !pairs::same_field(in.field, i0.field) ||
        ((in.flags ^ i0.flags) & SWF_ADAPTIVE)) {
      set_error("swf_pair_matrix: every electron and positron must share the field, grid, time window and step control");
      return SWF_EINVAL;
    }
    for (int a = 0; a < 3; ++a) {
      if (i0.grid.n[a] != 1) continue;
      const bool ok = k < n_e ? in.p[a] == i0.p[a] : in.q[a] == -i0.p[a];
      if (!ok) {
        set_error("swf_pair_matrix: along a trivial axis every p must be equal and every q = -p");
        return SWF_EINVAL;
      }
    }
  }
  cudaSetDevice(ctx->device);
  cudaStream_t st = ctx->stream;
  const GridDesc g = make_grid(i0.grid);
  const long K = 4L * g.N;
  const size_t elem = prec == SWF_C64 ? 8 : 16;
  std::vector<FieldDesc> fdU(n_e), fdV(n_p);
  std::vector<pairs::Wave> wu(n_e), wv(n_p);
  for (int m = 0; m < n_e; ++m) {
    fdU[m] = make_field_desc(electrons[m], 0);
    spinor_uv(electrons[m].p, electrons[m].s, false, wu[m].w);
    for (int a = 0; a < 3; ++a) wu[m].mom[a] = electrons[m].p[a];
    wu[m].sgn = 1.0;
  }
  for (int n = 0; n < n_p; ++n) {
    fdV[n] = make_field_desc(positrons[n], 1);
    spinor_uv(positrons[n].q, positrons[n].r, true, wv[n].w);
    for (int a = 0; a < 3; ++a) wv[n].mom[a] = positrons[n].q[a];
    wv[n].sgn = -1.0;
  }
  void *psiU, *psiV, *specU, *specV, *xU, *xV, *wU, *wV, *proj, *normU, *normV, *Cm, *Am, *BDm, *pw, *pku, *pres;
  if ((s = ws_get(ctx, "pairs.psiU", (size_t)n_e * K * elem, &psiU)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "pairs.psiV", (size_t)n_p * K * elem, &psiV)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "pairs.specU", (size_t)n_e * K * 16, &specU)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "pairs.specV", (size_t)n_p * K * 16, &specV)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "pairs.xU", (size_t)n_e * K * 16, &xU)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "pairs.xV", (size_t)n_p * K * 16, &xV)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "pairs.waveU", (size_t)n_e * K * 16, &wU)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "pairs.waveV", (size_t)n_p * K * 16, &wV)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "pairs.proj", (size_t)2 * n_e * K * 16, &proj)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "pairs.normU", (size_t)n_e * 8, &normU)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "pairs.normV", (size_t)n_p * 8, &normV)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "pairs.C", (size_t)n_e * n_p * 16, &Cm)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "pairs.A", (size_t)n_e * n_p * 16, &Am)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "pairs.BD", (size_t)2 * n_e * n_p * 16, &BDm)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "pairs.waves", sizeof(pairs::Wave) * (size_t)(n_e + n_p), &pw)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "pairs.Ku", 3 * sizeof(double), &pku)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "pairs.results", sizeof(swf_result) * (size_t)n_e * n_p, &pres)) != SWF_OK) return s;
  // one march per electron (U waves) and per positron (V waves), then their FP64 transforms
  const double t_in = i0.grid.t_in;
  const int adaptive = (i0.flags & SWF_ADAPTIVE) ? 1 : 0;
  if ((s = march_fields(ctx, g, t_in, i0.grid.t_out, i0.grid.n_steps, n_e, fdU.data(), prec, psiU, st, adaptive)) != SWF_OK)
    return s;
  if ((s = march_fields(ctx, g, t_in, i0.grid.t_out, i0.grid.n_steps, n_p, fdV.data(), prec, psiV, st, adaptive)) != SWF_OK)
    return s;
  if ((s = transform_fields(ctx, g, n_e, prec, psiU, (double2*)specU, st)) != SWF_OK) return s;
  if ((s = transform_fields(ctx, g, n_p, prec, psiV, (double2*)specV, st)) != SWF_OK) return s;
  if ((s = field_norms(ctx, g, n_e, prec, psiU, (double*)normU, st)) != SWF_OK) return s;
  if ((s = field_norms(ctx, g, n_p, prec, psiV, (double*)normV, st)) != SWF_OK) return s;
  cudaError_t e = cudaMemcpyAsync(pw, wu.data(), sizeof(pairs::Wave) * n_e, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync((pairs::Wave*)pw + n_e, wv.data(), sizeof(pairs::Wave) * n_p, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pku, fdU[0].K, 3 * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "upload pair tables");
  const int gx = (int)std::min<long>((g.N + 255) / 256, 1024);
  {
    ProfScope ps(ctx, "k_widen", st);
    const size_t nu = (size_t)n_e * K, nv = (size_t)n_p * K;
    const int bu = (int)std::min<size_t>((nu + 255) / 256, 8192), bv = (int)std::min<size_t>((nv + 255) / 256, 8192);
    if (prec == SWF_C64) {
      pairs::k_widen<float><<<bu, 256, 0, st>>>((const cpx<float>*)psiU, (cpx<double>*)xU, nu);
      pairs::k_widen<float><<<bv, 256, 0, st>>>((const cpx<float>*)psiV, (cpx<double>*)xV, nv);
    } else {
      pairs::k_widen<double><<<bu, 256, 0, st>>>((const cpx<double>*)psiU, (cpx<double>*)xU, nu);
      pairs::k_widen<double><<<bv, 256, 0, st>>>((const cpx<double>*)psiV, (cpx<double>*)xV, nv);
    }
  }
  {
    ProfScope ps(ctx, "k_plane_waves", st);
    pairs::k_plane_waves<<<dim3(gx, n_e), 256, 0, st>>>((const pairs::Wave*)pw, g, t_in, (cpx<double>*)wU);
    pairs::k_plane_waves<<<dim3(gx, n_p), 256, 0, st>>>((const pairs::Wave*)pw + n_e, g, t_in, (cpx<double>*)wV);
  }
  {
    ProfScope ps(ctx, "k_project", st);
    pairs::k_project<<<dim3(gx, n_e), 256, 0, st>>>((const cpx<double>*)specU, g, (const double*)pku, n_e,
                                                    (cpx<double>*)proj);
  }
  double vol = 1.0;
  for (int a = 0; a < 3; ++a)
    if (g.n[a] > 1) vol *= g.L[a];
  const double cell = g.dx[0] * g.dx[1] * g.dx[2];
  if ((s = pairs::gemm_cn(ctx, (const cpx<double>*)xU, (const cpx<double>*)wV, n_e, n_p, K, cell, (cpx<double>*)Cm,
                          "pair overlaps C", st)) != SWF_OK)
    return s;
  if ((s = pairs::gemm_cn(ctx, (const cpx<double>*)wU, (const cpx<double>*)xV, n_e, n_p, K, cell, (cpx<double>*)Am,
                          "pair overlaps A", st)) != SWF_OK)
    return s;
  if ((s = pairs::gemm_cn(ctx, (const cpx<double>*)proj, (const cpx<double>*)specV, 2 * n_e, n_p, K, 1.0 / vol,
                          (cpx<double>*)BDm, "pair overlaps B, D", st)) != SWF_OK)
    return s;
  {
    ProfScope ps(ctx, "k_pair_results", st);
    pairs::k_pair_results<<<(n_e * n_p + 255) / 256, 256, 0, st>>>((const cpx<double>*)Cm, (const cpx<double>*)Am,
                                                                   (const cpx<double>*)BDm, (const double*)normU,
                                                                   (const double*)normV, n_e, n_p, (swf_result*)pres);
  }
  e = cudaMemcpyAsync(results, pres, sizeof(swf_result) * (size_t)n_e * n_p, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_status(e, "download pair results");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "pair matrix");
  return SWF_OK;
}
