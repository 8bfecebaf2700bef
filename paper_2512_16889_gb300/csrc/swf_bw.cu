// Breit-Wheeler amplitude at t_in (Sec. IV): the analytic past terms of Eqs. 25-27 built with
// the energy projectors of Eq. 23, added to the finite-time terms integrated during the march
// (Eqs. 17, 33-35), in FP64.
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
  double Ku[3], Kv[3];
};

// One block per instance.  U~ = spec[2i], V~ = spec[2i+1] (continuum-normalised transforms at
// t_in); tat[2i] = U~(k - q) and tat[2i+1] = V~(p - k) by direct sums; macc = M(t_in) of the
// appended integral; norms[2i], norms[2i+1] = ||U_scat||^2, ||V_scat||^2.
__global__ void __launch_bounds__(256) k_bw_finalize(const BwInst* bi, GridDesc g, double t_in,
                                                     const cpx<double>* spec, const cpx<double>* tat,
                                                     const cpx<double>* macc, const double* norms,
                                                     swf_result* res) {
  __shared__ cpx<double> red[8];
  const int inst = blockIdx.x;
  const BwInst& I = bi[inst];
  const double k0 = sqrt(I.k[0] * I.k[0] + I.k[1] * I.k[1] + I.k[2] * I.k[2]);
  const cpx<double>* su = spec + (size_t)(2 * inst) * 4 * g.N;
  const cpx<double>* sv = spec + (size_t)(2 * inst + 1) * 4 * g.N;
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
        acc = acc + div_i(d, sg * Eu - sgp * Ev - k0);
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
  o.diag[0] = norms[2 * inst];
  o.diag[1] = norms[2 * inst + 1];
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

size_t bw_inst_size() { return sizeof(BwInst); }

void bw_fill_inst(void* dst, const swf_instance& in, int out, const FieldDesc& fu, const FieldDesc& fv,
                  const int shift[3]) {
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
  *reinterpret_cast<BwInst*>(dst) = b;
}

}  // namespace swf
