// Breit-Wheeler amplitude at t_in (Sec. IV), in FP64: the analytic past terms of Eqs. 25-27 built
// with the energy projectors of Eq. 23, added to the finite-time terms integrated during the march
// (Eqs. 17, 34-35); or the three terms of the partial-integration form (Eqs. 30-33) from the
// accumulators of that march.
#include "swf_internal.h"

namespace swf {

namespace {

// v <- (alpha . eps) v for a real polarisation (Dirac representation).
__device__ __forceinline__ void alpha_eps_d(const double* e, const cpx<double>* v, cpx<double>* o) {
  o[0] = e[2] * v[2] + e[0] * v[3] + e[1] * mul_mi(v[3]);
  o[1] = e[0] * v[2] + e[1] * mul_i(v[2]) - e[2] * v[3];
  o[2] = e[2] * v[0] + e[0] * v[1] + e[1] * mul_mi(v[1]);
  o[3] = e[0] * v[0] + e[1] * mul_i(v[0]) - e[2] * v[1];
}

// o = H0(kappa) v = (alpha.kappa + beta) v
__device__ __forceinline__ void h0_d(const double* k, const cpx<double>* v, cpx<double>* o) {
  alpha_eps_d(k, v, o);
  o[0] = o[0] + v[0];
  o[1] = o[1] + v[1];
  o[2] = o[2] - v[2];
  o[3] = o[3] - v[3];
}

// o = P_sign(kappa) v = (v + sign H0 v / E) / 2: positive (sign = +1, evolves as e^{-iEt}) or
// negative (sign = -1) energy part.
__device__ __forceinline__ void proj_d(const double* k, int sign, const cpx<double>* v, cpx<double>* o) {
  cpx<double> hv[4];
  h0_d(k, v, hv);
  const double E = sqrt(1.0 + k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
  for (int a = 0; a < 4; ++a) o[a] = 0.5 * (v[a] + (sign / E) * hv[a]);
}

__device__ __forceinline__ cpx<double> div_i(cpx<double> a, double om) {  // a / (i om)
  return mk<double>(a.y / om, -a.x / om);
}

}  // namespace

struct BwInst {
  double p[3], q[3], k[3], eps[3];
  int s, r;
  int out;
  int shift[3];   // the photon momentum in grid modes per non-trivial axis
  int src;        // the marched pair (U, V) of this amplitude: spectra and norms at index src
  double Ku[3], Kv[3];
};

// One block per amplitude i (an instance, or one photon of a photon scan).  With c = bi[i].src:
// U~ = spec[2c], V~ = spec[2c+1] (continuum-normalised transforms at t_in); tat[2i] = U~(k - q)
// and tat[2i+1] = V~(p - k) by direct sums; macc = M(t_in) of the appended integral; norms[2c],
// norms[2c+1] = ||U_scat||^2, ||V_scat||^2.
__global__ void __launch_bounds__(256) k_bw_finalize(const BwInst* bi, GridDesc g, double t_in,
                                                     const cpx<double>* spec, const cpx<double>* tat,
                                                     const cpx<double>* macc, const double* norms,
                                                     swf_result* res) {
  __shared__ cpx<double> red[8];
  const int inst = blockIdx.x;
  const BwInst& I = bi[inst];
  const double k0 = sqrt(I.k[0] * I.k[0] + I.k[1] * I.k[1] + I.k[2] * I.k[2]);
  const cpx<double>* su = spec + (size_t)(2 * I.src) * 4 * g.N;
  const cpx<double>* sv = spec + (size_t)(2 * I.src + 1) * 4 * g.N;
  // scat, scat: sum over U modes kappa, V mode kappa - k (periodic), both energy signs each
  cpx<double> acc = mk<double>(0, 0);
  for (int j = threadIdx.x; j < g.N; j += blockDim.x) {
    const int ix = j % g.n[0];
    const int iy = (j / g.n[0]) % g.n[1];
    const int iz = j / (g.n[0] * g.n[1]);
    const int id[3] = {ix, iy, iz};
    double ku[3], kv[3];
    int jv[3];
    for (int a = 0; a < 3; ++a) {
      jv[a] = ((id[a] - I.shift[a]) % g.n[a] + g.n[a]) % g.n[a];
      ku[a] = g.n[a] > 1 ? mode_kappa(id[a], g.n[a], g.L[a]) : I.Ku[a];
      kv[a] = g.n[a] > 1 ? mode_kappa(jv[a], g.n[a], g.L[a]) : I.Kv[a];
    }
    const int j2 = (jv[2] * g.n[1] + jv[1]) * g.n[0] + jv[0];
    // the grid sum of the pair's plane waves, N e^{i(kappa_v + k - kappa_u).x0}: -1 for a V mode
    // that wrapped around an odd axis length (an odd number of times), 1 otherwise
    int odd = 0;
    for (int a = 0; a < 3; ++a) {
      if (g.n[a] > 1 && (g.n[a] & 1)) {
        const long fu = id[a] < (g.n[a] + 1) / 2 ? id[a] : id[a] - g.n[a];
        const long fv = jv[a] < (g.n[a] + 1) / 2 ? jv[a] : jv[a] - g.n[a];
        odd ^= (int)(((fu - fv - I.shift[a]) / g.n[a]) & 1);
      }
    }
    const double wrap = odd ? -1.0 : 1.0;
    cpx<double> u[4], v[4];
    for (int a = 0; a < 4; ++a) {
      u[a] = su[(size_t)a * g.N + j];
      v[a] = sv[(size_t)a * g.N + j2];
    }
    const double Eu = sqrt(1.0 + ku[0] * ku[0] + ku[1] * ku[1] + ku[2] * ku[2]);
    const double Ev = sqrt(1.0 + kv[0] * kv[0] + kv[1] * kv[1] + kv[2] * kv[2]);
    for (int sg = -1; sg <= 1; sg += 2) {
      cpx<double> pu[4];
      proj_d(ku, sg, u, pu);
      for (int sgp = -1; sgp <= 1; sgp += 2) {
        cpx<double> pv[4], apv[4];
        proj_d(kv, sgp, v, pv);
        alpha_eps_d(I.eps, pv, apv);
        cpx<double> d = mk<double>(0, 0);
        for (int a = 0; a < 4; ++a) d = d + cdot(pu[a], apv[a]);
        acc = acc + div_i(wrap * d, sg * Eu - sgp * Ev - k0);
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    acc.x += __shfl_down_sync(0xffffffffu, acc.x, off);
    acc.y += __shfl_down_sync(0xffffffffu, acc.y, off);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x != 0) return;
  cpx<double> ss = mk<double>(0, 0);
  for (int w = 0; w < 8; ++w) ss = ss + red[w];
  double vol = 1.0;
  for (int a = 0; a < 3; ++a)
    if (g.n[a] > 1) vol *= g.L[a];
  double sn, cs;
  sincos(-k0 * t_in, &sn, &cs);
  const cpx<double> ek = mk<double>(cs, sn);
  ss = (1.0 / vol) * (ek * ss);
  // back, scat: U_back = u_s(p) e^{-i p0 t} in mode p; V_scat needed at p - k
  double sp[8];
  spinor_uv(I.p, I.s, false, sp);
  cpx<double> ub[4], vv[4], pv[4], apv[4];
  for (int a = 0; a < 4; ++a) { ub[a] = mk<double>(sp[2 * a], sp[2 * a + 1]); vv[a] = tat[4 * (2 * inst + 1) + a]; }
  double kv[3];
  for (int a = 0; a < 3; ++a) kv[a] = I.p[a] - I.k[a];
  const double p0 = energy3(I.p), Ekv = energy3(kv);
  cpx<double> bs = mk<double>(0, 0);
  for (int sgp = -1; sgp <= 1; sgp += 2) {
    proj_d(kv, sgp, vv, pv);
    alpha_eps_d(I.eps, pv, apv);
    cpx<double> d = mk<double>(0, 0);
    for (int a = 0; a < 4; ++a) d = d + cdot(ub[a], apv[a]);
    bs = bs + div_i(d, p0 - sgp * Ekv - k0);
  }
  sincos(p0 * t_in, &sn, &cs);
  bs = ek * (mk<double>(cs, sn) * bs);
  // scat, back: V_back = v_r(q) e^{+i q0 t} in mode -q; U_scat needed at k - q
  spinor_uv(I.q, I.r, true, sp);
  cpx<double> vb[4], uu[4], pu[4], avb[4];
  for (int a = 0; a < 4; ++a) { vb[a] = mk<double>(sp[2 * a], sp[2 * a + 1]); uu[a] = tat[4 * (2 * inst) + a]; }
  alpha_eps_d(I.eps, vb, avb);
  double ku[3];
  for (int a = 0; a < 3; ++a) ku[a] = I.k[a] - I.q[a];
  const double q0 = energy3(I.q), Eku = energy3(ku);
  cpx<double> sb = mk<double>(0, 0);
  for (int sg = -1; sg <= 1; sg += 2) {
    proj_d(ku, sg, uu, pu);
    cpx<double> d = mk<double>(0, 0);
    for (int a = 0; a < 4; ++a) d = d + cdot(pu[a], avb[a]);
    sb = sb + div_i(d, sg * Eku + q0 - k0);
  }
  sincos(q0 * t_in, &sn, &cs);
  sb = ek * (mk<double>(cs, sn) * sb);
  // M_finite = -M(t_in) of the appended integral
  const cpx<double> t_ss = ss - macc[3 * inst], t_bs = bs - macc[3 * inst + 1], t_sb = sb - macc[3 * inst + 2];
  const cpx<double> M = t_ss + t_bs + t_sb;
  swf_result& o = res[I.out];
  o.amp[0] = t_ss.x; o.amp[1] = t_ss.y;
  o.amp[2] = t_bs.x; o.amp[3] = t_bs.y;
  o.amp[4] = t_sb.x; o.amp[5] = t_sb.y;
  o.amp[6] = M.x; o.amp[7] = M.y;
  o.prob[0] = M.x * M.x + M.y * M.y;
  o.prob[1] = 0.0;
  o.diag[0] = norms[2 * I.src];
  o.diag[1] = norms[2 * I.src + 1];
}

swf_status bw_finalize(swf_ctx* ctx, const GridDesc& g, int n_inst, const void* bw_host, double t_in,
                       const double2* spec, const double2* tat, const double2* macc, const double* norms,
                       swf_result* results, cudaStream_t st) {
  void* pb;
  swf_status s = ws_get(ctx, "bw.inst", sizeof(BwInst) * n_inst, &pb);
  if (s != SWF_OK) return s;
  cudaError_t e = cudaMemcpyAsync(pb, bw_host, sizeof(BwInst) * n_inst, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "upload Breit-Wheeler table");
  {
    ProfScope ps(ctx, "k_bw_finalize", st);
    k_bw_finalize<<<n_inst, 256, 0, st>>>((const BwInst*)pb, g, t_in, (const cpx<double>*)spec,
                                          (const cpx<double>*)tat, (const cpx<double>*)macc, norms, results);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "Breit-Wheeler finalize");
  return SWF_OK;
}

// Partial-integration form (Eqs. 30-33): one thread per instance turns the march's accumulators
// macc[inst] = (mode sum of the ss integrand, D_U[4], D_V[4]) into the three terms.  With the
// march's weights w_i = h b_i (h < 0) every term is M = -sum_i w_i M-dot(t_i):
//   M_ss = -i dx^{2d} e^{i k.x0} / L^d * (mode sum)            (x0: the grid origin)
//   M_bs = -i dx^d sum_s' u^+ (alpha.eps) P_s'(p - k) D_V / (p0 - s' E(p - k) - k0)
//   M_sb = -i dx^d D_U^+ sum_s P_s(k - q) (alpha.eps) v / (s E(k - q) + q0 - k0)
__global__ void k_bw_finalize_partial(const BwInst* bi, GridDesc g, const cpx<double>* macc, const double* norms,
                                      swf_result* res) {
  if (threadIdx.x != 0) return;
  const int inst = blockIdx.x;
  const BwInst& I = bi[inst];
  const cpx<double>* m = macc + 9 * inst;
  const double k0 = sqrt(I.k[0] * I.k[0] + I.k[1] * I.k[1] + I.k[2] * I.k[2]);
  double vol = 1.0, kx0 = 0.0;
  for (int a = 0; a < 3; ++a)
    if (g.n[a] > 1) {
      vol *= g.L[a];
      kx0 += I.k[a] * g.x0[a];
    }
  const double cell = g.dx[0] * g.dx[1] * g.dx[2];
  double sn, cs;
  sincos(kx0, &sn, &cs);
  const cpx<double> t_ss = mul_mi((cell * cell / vol) * (mk<double>(cs, sn) * m[0]));
  // back, scat
  double sp[8];
  spinor_uv(I.p, I.s, false, sp);
  cpx<double> ub[4], dv[4], pv[4], apv[4];
  for (int a = 0; a < 4; ++a) {
    ub[a] = mk<double>(sp[2 * a], sp[2 * a + 1]);
    dv[a] = m[5 + a];
  }
  double kv[3];
  for (int a = 0; a < 3; ++a) kv[a] = I.p[a] - I.k[a];
  const double p0 = energy3(I.p), Ekv = energy3(kv);
  cpx<double> bs = mk<double>(0, 0);
  for (int sgp = -1; sgp <= 1; sgp += 2) {
    proj_d(kv, sgp, dv, pv);
    alpha_eps_d(I.eps, pv, apv);
    cpx<double> d = mk<double>(0, 0);
    for (int a = 0; a < 4; ++a) d = d + cdot(ub[a], apv[a]);
    bs = bs + (1.0 / (p0 - sgp * Ekv - k0)) * d;
  }
  const cpx<double> t_bs = mul_mi(cell * bs);
  // scat, back
  spinor_uv(I.q, I.r, true, sp);
  cpx<double> vb[4], avb[4], pw[4], wsb[4];
  for (int a = 0; a < 4; ++a) {
    vb[a] = mk<double>(sp[2 * a], sp[2 * a + 1]);
    wsb[a] = mk<double>(0, 0);
  }
  alpha_eps_d(I.eps, vb, avb);
  double ku[3];
  for (int a = 0; a < 3; ++a) ku[a] = I.k[a] - I.q[a];
  const double q0 = energy3(I.q), Eku = energy3(ku);
  for (int sg = -1; sg <= 1; sg += 2) {
    proj_d(ku, sg, avb, pw);
    for (int a = 0; a < 4; ++a) wsb[a] = wsb[a] + (1.0 / (sg * Eku + q0 - k0)) * pw[a];
  }
  cpx<double> sb = mk<double>(0, 0);
  for (int a = 0; a < 4; ++a) sb = sb + cdot(m[1 + a], wsb[a]);
  const cpx<double> t_sb = mul_mi(cell * sb);
  const cpx<double> M = t_ss + t_bs + t_sb;
  swf_result& o = res[I.out];
  o.amp[0] = t_ss.x; o.amp[1] = t_ss.y;
  o.amp[2] = t_bs.x; o.amp[3] = t_bs.y;
  o.amp[4] = t_sb.x; o.amp[5] = t_sb.y;
  o.amp[6] = M.x; o.amp[7] = M.y;
  o.prob[0] = M.x * M.x + M.y * M.y;
  o.prob[1] = 0.0;
  o.diag[0] = norms[2 * I.src];
  o.diag[1] = norms[2 * I.src + 1];
}

swf_status bw_finalize_partial(swf_ctx* ctx, const GridDesc& g, int n_inst, const void* bw_host,
                               const double2* macc, const double* norms, swf_result* results, cudaStream_t st) {
  void* pb;
  swf_status s = ws_get(ctx, "bw.inst", sizeof(BwInst) * n_inst, &pb);
  if (s != SWF_OK) return s;
  cudaError_t e = cudaMemcpyAsync(pb, bw_host, sizeof(BwInst) * n_inst, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "upload Breit-Wheeler table");
  {
    ProfScope ps(ctx, "k_bw_finalize_partial", st);
    k_bw_finalize_partial<<<n_inst, 32, 0, st>>>((const BwInst*)pb, g, (const cpx<double>*)macc, norms, results);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "Breit-Wheeler finalize (partial integration)");
  return SWF_OK;
}

// Photon wave packet sampled on grid momenta (Sec. IV, closing paragraphs): by linearity in the
// photon wave function its amplitude is sum_j w_j M(k_j, eps_j).  One thread adds the n amplitudes
// (per term and in total) in order.
__global__ void k_bw_packet(const swf_result* res, int n, const double* w, cpx<double>* out) {
  if (threadIdx.x != 0) return;
  cpx<double> acc[4] = {mk<double>(0, 0), mk<double>(0, 0), mk<double>(0, 0), mk<double>(0, 0)};
  for (int j = 0; j < n; ++j) {
    const cpx<double> wj = mk<double>(w[2 * j], w[2 * j + 1]);
    for (int c = 0; c < 4; ++c) acc[c] = acc[c] + wj * mk<double>(res[j].amp[2 * c], res[j].amp[2 * c + 1]);
  }
  for (int c = 0; c < 4; ++c) out[c] = acc[c];
}

swf_status bw_packet(swf_ctx* ctx, int n, const swf_result* results, const double* weights_host, double2* out,
                     cudaStream_t st) {
  void* pw;
  swf_status s = ws_get(ctx, "bw.packet_w", sizeof(double) * 2 * (size_t)n, &pw);
  if (s != SWF_OK) return s;
  cudaError_t e = cudaMemcpyAsync(pw, weights_host, sizeof(double) * 2 * (size_t)n, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "upload packet weights");
  {
    ProfScope ps(ctx, "k_bw_packet", st);
    k_bw_packet<<<1, 32, 0, st>>>(results, n, (const double*)pw, (cpx<double>*)out);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "photon packet sum");
  return SWF_OK;
}

size_t bw_inst_size() { return sizeof(BwInst); }

void bw_fill_inst(void* dst, const swf_instance& in, int out, const FieldDesc& fu, const FieldDesc& fv,
                  const int shift[3], int src) {
  BwInst b;
  for (int a = 0; a < 3; ++a) {
    b.p[a] = in.p[a];
    b.q[a] = in.q[a];
    b.k[a] = in.k[a];
    b.eps[a] = in.eps[a];
    b.shift[a] = shift[a];
    b.Ku[a] = fu.K[a];
    b.Kv[a] = fv.K[a];
  }
  b.s = in.s;
  b.r = in.r;
  b.out = out;
  b.src = src;
  *reinterpret_cast<BwInst*>(dst) = b;
}

}  // namespace swf
