// C ABI of the SWF solver: context, validation, workspace and the orchestration of
// march -> projections -> per-instance results (Sec. II Eqs. 6-9, Sec. IV).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <tuple>
#include <vector>

#include "swf_internal.h"

namespace swf {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

swf_status cuda_status(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return SWF_ECUDA;
}

swf_status ws_get(swf_ctx* ctx, const std::string& name, size_t bytes, void** ptr) {
  if (bytes == 0) bytes = 16;
  auto it = ctx->ws.bufs.find(name);
  if (it != ctx->ws.bufs.end() && it->second.second >= bytes) {
    *ptr = it->second.first;
    return SWF_OK;
  }
  size_t old = it != ctx->ws.bufs.end() ? it->second.second : 0;
  if (ctx->ws.limit && ctx->ws.total - old + bytes > ctx->ws.limit) {
    set_error("workspace limit exceeded by buffer '" + name + "'");
    return SWF_ENOMEM;
  }
  if (it != ctx->ws.bufs.end()) {
    cudaFree(it->second.first);  // synchronises the device before the memory is reused
    ctx->ws.total -= old;
    ctx->ws.bufs.erase(it);
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc of " + std::to_string(bytes) + " bytes for '" + name + "' failed");
    return SWF_ENOMEM;
  }
  ctx->ws.bufs[name] = {p, bytes};
  ctx->ws.total += bytes;
  *ptr = p;
  return SWF_OK;
}

swf_status twiddles(swf_ctx* ctx, int n, int is_double, const void** ptr) {
  auto key = std::make_pair(n, is_double);
  auto it = ctx->tw.tables.find(key);
  if (it != ctx->tw.tables.end()) {
    *ptr = it->second;
    return SWF_OK;
  }
  std::vector<double> re(n), im(n);
  for (int m = 0; m < n; ++m) {
    // exp(-2 pi i m/n) evaluated in long double and rounded once
    long double a = -2.0L * 3.14159265358979323846264338327950288L * (long double)m / (long double)n;
    re[m] = (double)cosl(a);
    im[m] = (double)sinl(a);
  }
  void* p = nullptr;
  size_t bytes = (size_t)n * (is_double ? 16 : 8);
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) return cuda_status(e, "cudaMalloc(twiddles)");
  std::vector<unsigned char> host(bytes);
  for (int m = 0; m < n; ++m) {
    if (is_double) {
      double v[2] = {re[m], im[m]};
      std::memcpy(&host[16 * m], v, 16);
    } else {
      float v[2] = {(float)re[m], (float)im[m]};
      std::memcpy(&host[8 * m], v, 8);
    }
  }
  e = cudaMemcpy(p, host.data(), bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_status(e, "upload twiddles");
  ctx->tw.tables[key] = p;
  *ptr = p;
  return SWF_OK;
}

int prof_begin(swf_ctx* ctx, const char* family, cudaStream_t st) {
  Profiler& P = ctx->prof;
  ++P.launches;
  if (!P.on) return -1;
  if (P.used + 2 > P.pool.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t ev;
      if (cudaEventCreate(&ev) != cudaSuccess) { cudaGetLastError(); return -1; }
      P.pool.push_back(ev);
    }
  }
  int fam = -1;
  for (size_t i = 0; i < P.families.size(); ++i)
    if (P.families[i] == family) fam = (int)i;
  if (fam < 0) { P.families.push_back(family); fam = (int)P.families.size() - 1; }
  const size_t first = P.used;
  P.used += 2;
  cudaEventRecord(P.pool[first], st);
  P.marks.push_back({fam, first});
  return (int)P.marks.size() - 1;
}

void prof_end(swf_ctx* ctx, int mark, cudaStream_t st) {
  if (mark < 0) return;
  Profiler& P = ctx->prof;
  cudaEventRecord(P.pool[P.marks[mark].second + 1], st);
}

bool make_radix_plan(int n, RadixPlan* pl) {
  pl->n = n;
  pl->npass = 0;
  int m = n;
  while (m % 4 == 0 && pl->npass < 12) { pl->rad[pl->npass++] = 4; m /= 4; }
  while (m % 2 == 0 && pl->npass < 12) { pl->rad[pl->npass++] = 2; m /= 2; }
  while (m % 3 == 0 && pl->npass < 12) { pl->rad[pl->npass++] = 3; m /= 3; }
  while (m % 5 == 0 && pl->npass < 12) { pl->rad[pl->npass++] = 5; m /= 5; }
  return m == 1;
}

GridDesc make_grid(const swf_grid& g) {
  GridDesc d;
  d.N = 1;
  for (int a = 0; a < 3; ++a) {
    d.n[a] = g.n[a];
    d.L[a] = g.L[a];
    d.N *= g.n[a];
    d.dx[a] = g.n[a] > 1 ? g.L[a] / g.n[a] : 1.0;
    d.x0[a] = g.n[a] > 1 ? -0.5 * g.L[a] : 0.0;
  }
  return d;
}

FieldDesc make_field_desc(const swf_instance& in, int bg) {
  FieldDesc f;
  std::memset(&f, 0, sizeof f);
  f.kind = in.field.kind;
  for (int i = 0; i < 8; ++i) f.prm[i] = in.field.prm[i];
  switch (in.field.kind) {
    case SWF_FIELD_SAUTER_GAUSS:
    case SWF_FIELD_PULSE_GAUSS: f.acomp = 1; break;
    case SWF_FIELD_SINGLE_E:
    case SWF_FIELD_DOUBLE_E: f.acomp = 0; break;
    default: f.acomp = -1;
  }
  double mom[3];
  for (int a = 0; a < 3; ++a) mom[a] = bg == 0 ? in.p[a] : in.q[a];
  spinor_uv(mom, bg == 0 ? in.s : in.r, bg == 1, f.w);
  f.e0 = energy3(mom);
  f.tsign = bg == 0 ? -1.0 : 1.0;
  for (int a = 0; a < 3; ++a) {
    f.pmom[a] = bg == 0 ? mom[a] : -mom[a];
    f.K[a] = in.grid.n[a] == 1 ? f.pmom[a] : 0.0;
  }
  return f;
}

// ------------------------------------------------------------------ validation
static bool finite3(const double* v) { return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]); }

static swf_status validate(int n_inst, const swf_instance* inst, swf_process process, swf_precision prec) {
  if (n_inst < 0) { set_error("n_inst < 0"); return SWF_EINVAL; }
  if (n_inst > 0 && !inst) { set_error("instances pointer is NULL"); return SWF_EINVAL; }
  if (prec != SWF_C64 && prec != SWF_C128) { set_error("unknown precision"); return SWF_EINVAL; }
  if (process != SWF_SCHWINGER && process != SWF_BREIT_WHEELER) { set_error("unknown process"); return SWF_EINVAL; }
  for (int i = 0; i < n_inst; ++i) {
    const swf_instance& in = inst[i];
    char pre[64];
    std::snprintf(pre, sizeof pre, "instance %d: ", i);
    long long N = 1;
    for (int a = 0; a < 3; ++a) {
      const int n = in.grid.n[a];
      RadixPlan pl;
      if (n < 1 || n > 512 || !make_radix_plan(n, &pl)) {
        set_error(std::string(pre) + "each n must be in [1, 512] and factor into 2, 3, 5");
        return SWF_EINVAL;
      }
      if (n > 1 && !(in.grid.L[a] > 0.0 && std::isfinite(in.grid.L[a]))) {
        set_error(std::string(pre) + "box length must be positive on non-trivial axes");
        return SWF_EINVAL;
      }
      N *= n;
    }
    if (in.grid.n_steps < 1) { set_error(std::string(pre) + "n_steps must be >= 1"); return SWF_EINVAL; }
    if (!(in.grid.t_in < in.grid.t_out) || !std::isfinite(in.grid.t_in) || !std::isfinite(in.grid.t_out)) {
      set_error(std::string(pre) + "need finite t_in < t_out");
      return SWF_EINVAL;
    }
    if (in.field.kind < SWF_FIELD_ZERO || in.field.kind > SWF_FIELD_DOUBLE_E) {
      set_error(std::string(pre) + "unknown field kind");
      return SWF_EINVAL;
    }
    for (int k = 0; k < 8; ++k)
      if (!std::isfinite(in.field.prm[k])) { set_error(std::string(pre) + "field parameters must be finite"); return SWF_EINVAL; }
    const double* prm = in.field.prm;
    if ((in.field.kind == SWF_FIELD_SAUTER_GAUSS && prm[1] == 0.0) ||
        (in.field.kind == SWF_FIELD_PULSE_GAUSS && (prm[2] == 0.0 || prm[3] == 0.0)) ||
        ((in.field.kind == SWF_FIELD_SINGLE_E || in.field.kind == SWF_FIELD_DOUBLE_E) && prm[2] == 0.0)) {
      set_error(std::string(pre) + "a field width or frequency is zero");
      return SWF_EINVAL;
    }
    if ((in.s != 1 && in.s != -1) || (in.r != 1 && in.r != -1)) {
      set_error(std::string(pre) + "spins must be +1 or -1");
      return SWF_EINVAL;
    }
    if (!finite3(in.p) || !finite3(in.q) || !finite3(in.k) || !finite3(in.eps)) {
      set_error(std::string(pre) + "momenta must be finite");
      return SWF_EINVAL;
    }
  }
  return SWF_OK;
}

swf_status validate_instances(int n_inst, const swf_instance* inst, swf_precision prec) {
  return validate(n_inst, inst, SWF_SCHWINGER, prec);
}

static cudaStream_t pick_stream(swf_ctx* ctx, void* stream) {
  return stream ? (cudaStream_t)stream : ctx->stream;
}

// ------------------------------------------------------------------ per-instance results
struct InstDev {
  double p[3];
  double q[3];
  int s, r;
  int out;      // index in the results array
  int full;     // both lines of Eq. 8
  double Ku[3];  // trivial-axis momentum of the electron wave
};

// One block per instance: C, A, B, D and both lines of Eq. 8 (B and D as sums over the grid
// modes with the energy projectors, sum_s' u u^+ = P_+ and sum_s' v v^+ = P_-).
__global__ void __launch_bounds__(256) k_finalize(const InstDev* id, GridDesc g, double t_in,
                                                  const cpx<double>* specU, const cpx<double>* specV,
                                                  const cpx<double>* uq, const cpx<double>* vp,
                                                  const double* normU, const double* normV,
                                                  swf_result* res) {
  __shared__ cpx<double> red[8][2];
  const int f = blockIdx.x;
  const InstDev& I = id[f];
  cpx<double> accB = mk<double>(0, 0), accD = mk<double>(0, 0);
  if (I.full) {
    const cpx<double>* u = specU + (size_t)f * 4 * g.N;
    const cpx<double>* v = specV + (size_t)f * 4 * g.N;
    for (int j = threadIdx.x; j < g.N; j += blockDim.x) {
      const int ix = j % g.n[0];
      const int iy = (j / g.n[0]) % g.n[1];
      const int iz = j / (g.n[0] * g.n[1]);
      const double kx = g.n[0] > 1 ? mode_kappa(ix, g.n[0], g.L[0]) : I.Ku[0];
      const double ky = g.n[1] > 1 ? mode_kappa(iy, g.n[1], g.L[1]) : I.Ku[1];
      const double kz = g.n[2] > 1 ? mode_kappa(iz, g.n[2], g.L[2]) : I.Ku[2];
      const double E = sqrt(1.0 + kx * kx + ky * ky + kz * kz);
      cpx<double> uv[4], vv[4], hv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) { uv[a] = u[(size_t)a * g.N + j]; vv[a] = v[(size_t)a * g.N + j]; }
      // hv = H0(kappa) vv
      const cpx<double> a0 = vv[0], a1 = vv[1], a2 = vv[2], a3 = vv[3];
      hv[0] = a0 + kz * a2 + kx * a3 + ky * mul_mi(a3);
      hv[1] = a1 + kx * a2 + ky * mul_i(a2) - kz * a3;
      hv[2] = kz * a0 + kx * a1 + ky * mul_mi(a1) - a2;
      hv[3] = kx * a0 + ky * mul_i(a0) - kz * a1 - a3;
      cpx<double> uv_v = mk<double>(0, 0), uv_hv = mk<double>(0, 0);
#pragma unroll
      for (int a = 0; a < 4; ++a) { uv_v = uv_v + cdot(uv[a], vv[a]); uv_hv = uv_hv + cdot(uv[a], hv[a]); }
      // U^+ P_+- V = (U^+V +- U^+ H0 V / E)/2
      accB = accB + 0.5 * (uv_v + (1.0 / E) * uv_hv);
      accD = accD + 0.5 * (uv_v - (1.0 / E) * uv_hv);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      accB.x += __shfl_down_sync(0xffffffffu, accB.x, off);
      accB.y += __shfl_down_sync(0xffffffffu, accB.y, off);
      accD.x += __shfl_down_sync(0xffffffffu, accD.x, off);
      accD.y += __shfl_down_sync(0xffffffffu, accD.y, off);
    }
    if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5][0] = accB; red[threadIdx.x >> 5][1] = accD; }
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  double vol = 1.0;
  for (int a = 0; a < 3; ++a)
    if (g.n[a] > 1) vol *= g.L[a];
  cpx<double> B = mk<double>(0, 0), D = mk<double>(0, 0);
  if (I.full) {
    for (int w = 0; w < 8; ++w) { B = B + red[w][0]; D = D + red[w][1]; }
    B = (1.0 / vol) * B;
    D = (1.0 / vol) * D;
  }
  // C = (U_scat | V_back(r, q)) = exp(i q0 t_in) conj(U~(-q)) . v_r(q)
  double sp[8];
  spinor_uv(I.q, I.r, true, sp);
  cpx<double> C = mk<double>(0, 0);
  for (int a = 0; a < 4; ++a) C = C + cdot(uq[4 * f + a], mk<double>(sp[2 * a], sp[2 * a + 1]));
  double sn, cs;
  sincos(energy3(I.q) * t_in, &sn, &cs);
  C = mk<double>(cs, sn) * C;
  // without the full pair number: C for the other positron spin as well
  cpx<double> C2 = mk<double>(0, 0);
  if (!I.full) {
    spinor_uv(I.q, -I.r, true, sp);
    for (int a = 0; a < 4; ++a) C2 = C2 + cdot(uq[4 * f + a], mk<double>(sp[2 * a], sp[2 * a + 1]));
    C2 = mk<double>(cs, sn) * C2;
  }
  cpx<double> A = mk<double>(0, 0);
  if (I.full) {
    // A = (U_back(s, p) | V_scat) = exp(i p0 t_in) u_s(p)^+ V~(p)
    spinor_uv(I.p, I.s, false, sp);
    for (int a = 0; a < 4; ++a) A = A + cdot(mk<double>(sp[2 * a], sp[2 * a + 1]), vp[4 * f + a]);
    sincos(energy3(I.p) * t_in, &sn, &cs);
    A = mk<double>(cs, sn) * A;
  }
  swf_result& o = res[I.out];
  o.amp[0] = C.x; o.amp[1] = C.y;
  if (I.full) {
    o.amp[2] = D.x; o.amp[3] = D.y;
  } else {
    o.amp[2] = C2.x; o.amp[3] = C2.y;
  }
  o.amp[4] = A.x; o.amp[5] = A.y;
  o.amp[6] = B.x; o.amp[7] = B.y;
  const cpx<double> CD = C + D, AB = A + B;
  o.prob[0] = CD.x * CD.x + CD.y * CD.y;
  o.prob[1] = I.full ? AB.x * AB.x + AB.y * AB.y : C2.x * C2.x + C2.y * C2.y;
  o.diag[0] = normU[f];
  o.diag[1] = (I.full && normV) ? normV[f] : 0.0;
}

struct GroupKey {
  int n[3];
  double L[3];
  double t_in, t_out;
  int n_steps;
  int full;
  int adaptive = 0;
  bool operator<(const GroupKey& o) const {
    return std::tie(n[0], n[1], n[2], L[0], L[1], L[2], t_in, t_out, n_steps, full, adaptive) <
           std::tie(o.n[0], o.n[1], o.n[2], o.L[0], o.L[1], o.L[2], o.t_in, o.t_out, o.n_steps, o.full, o.adaptive);
  }
};

// In the automatic mode a set of groups is marched together when all of them hold fewer fields x
// grid points than this (per evaluation): above it every group fills the GPU by itself and one
// launch sequence per group was as fast (Breit-Wheeler on the uneven grids, 300 steps: grouped
// +5 % at 8 instances, 2 per grid size; level at 16; -3 % at 32).
constexpr double kMultiAutoSites = 4.0 * 1024 * 1024;

// Time grid and non-trivial axes: groups that agree on these can be marched together.
struct MultiKey {
  double t_in, t_out;
  int n_steps, ny_on, nz_on;
  bool operator<(const MultiKey& o) const {
    return std::tie(t_in, t_out, n_steps, ny_on, nz_on) < std::tie(o.t_in, o.t_out, o.n_steps, o.ny_on, o.nz_on);
  }
};

// Marches, in multi-grid marches, the fields of every fixed-step Schwinger group that runs on the
// pass kernels and shares its time grid and non-trivial axes with another such group (at most
// eight groups per march).  premarched[group] = device buffer [F_U (+ F_V)][4][N] of the group's
// psi(t_in): the U fields, then (full pair number) the V fields.
static swf_status premarch_schwinger(swf_ctx* ctx, const swf_instance* inst,
                                     const std::map<GroupKey, std::vector<int>>& groups, swf_precision prec,
                                     std::map<const GroupKey*, void*>& premarched, cudaStream_t st) {
  if (!ctx->multi_grid) return SWF_OK;
  const size_t elem = prec == SWF_C64 ? 8 : 16;
  std::map<MultiKey, std::vector<const GroupKey*>> sets;
  std::map<const GroupKey*, std::vector<FieldDesc>> fds;
  for (auto& kv : groups) {
    if (kv.first.adaptive) continue;
    const std::vector<int>& idx = kv.second;
    const swf_instance& i0 = inst[idx[0]];
    const GridDesc g = make_grid(i0.grid);
    std::vector<FieldDesc> fd;
    for (int f : idx) fd.push_back(make_field_desc(inst[f], 0));
    if (ctx->use_fused && fused_applicable(g, (int)fd.size(), fd.data(), prec)) continue;
    if (kv.first.full) {
      for (int f : idx) fd.push_back(make_field_desc(inst[f], 1));
      if (ctx->use_fused && fused_applicable(g, (int)idx.size(), fd.data() + idx.size(), prec)) continue;
    }
    sets[MultiKey{i0.grid.t_in, i0.grid.t_out, i0.grid.n_steps, g.n[1] > 1, g.n[2] > 1}].push_back(&kv.first);
    fds[&kv.first] = std::move(fd);
  }
  swf_status s;
  int buf = 0;
  for (auto& kv : sets) {
    const std::vector<const GroupKey*>& list = kv.second;
    for (size_t b = 0; b + 1 < list.size(); b += 8) {
      const size_t e = std::min(list.size(), b + 8);
      double sites = 0.0;
      for (size_t i = b; i < e; ++i) sites += (double)fds[list[i]].size() * make_grid(inst[groups.at(*list[i])[0]].grid).N;
      if (ctx->multi_grid == 1 && sites >= kMultiAutoSites) continue;
      std::vector<MultiGroup> mg;
      for (size_t i = b; i < e; ++i) {
        const GroupKey* k = list[i];
        const std::vector<FieldDesc>& fd = fds[k];
        const GridDesc g = make_grid(inst[groups.at(*k)[0]].grid);
        void* out = nullptr;
        if ((s = ws_get(ctx, "solve.multi" + std::to_string(buf++), fd.size() * 4 * (size_t)g.N * elem, &out)) != SWF_OK)
          return s;
        mg.push_back(MultiGroup{g, (int)fd.size(), fd.data(), out, nullptr, nullptr});
        premarched[k] = out;
      }
      s = march_fields_multi(ctx, mg, kv.first.t_in, kv.first.t_out, kv.first.n_steps, prec, st);
      if (s == SWF_EUNSUPPORTED) {  // not a form the grouped launch takes: these groups march alone
        for (size_t i = b; i < e; ++i) premarched.erase(list[i]);
        continue;
      }
      if (s != SWF_OK) return s;
    }
  }
  return SWF_OK;
}

static swf_status solve_schwinger(swf_ctx* ctx, int n_inst, const swf_instance* inst, swf_precision prec,
                                  swf_result* results_dev, double* spectrum_dev, cudaStream_t st) {
  std::map<GroupKey, std::vector<int>> groups;
  std::vector<size_t> spec_off(n_inst, 0);
  size_t off = 0;
  for (int i = 0; i < n_inst; ++i) {
    const swf_instance& in = inst[i];
    GroupKey k;
    for (int a = 0; a < 3; ++a) { k.n[a] = in.grid.n[a]; k.L[a] = in.grid.n[a] > 1 ? in.grid.L[a] : 0.0; }
    k.t_in = in.grid.t_in;
    k.t_out = in.grid.t_out;
    k.n_steps = in.grid.n_steps;
    k.full = (in.flags & SWF_WANT_FULL_N) ? 1 : 0;
    k.adaptive = (in.flags & SWF_ADAPTIVE) ? 1 : 0;
    groups[k].push_back(i);
    if (in.flags & SWF_WANT_SPECTRUM) {
      spec_off[i] = off;
      off += (size_t)2 * in.grid.n[0] * in.grid.n[1] * in.grid.n[2];
    }
  }
  const size_t elem = prec == SWF_C64 ? 8 : 16;
  swf_status s;
  // groups on the pass kernels that share a time grid and their non-trivial axes: every march
  // of those groups (U, and V for the full pair number) in one multi-grid march
  std::map<const GroupKey*, void*> premarched;
  if ((s = premarch_schwinger(ctx, inst, groups, prec, premarched, st)) != SWF_OK) return s;
  for (auto& kv : groups) {
    const std::vector<int>& idx = kv.second;
    const int F = (int)idx.size();
    const swf_instance& i0 = inst[idx[0]];
    const GridDesc g = make_grid(i0.grid);
    const bool full = kv.first.full != 0;
    auto pre = premarched.find(&kv.first);
    std::vector<FieldDesc> fdU(F), fdV(F);
    std::vector<InstDev> idv(F);
    std::vector<double> kq(3 * F), kp(3 * F);
    bool any_spec = false;
    for (int f = 0; f < F; ++f) {
      const swf_instance& in = inst[idx[f]];
      fdU[f] = make_field_desc(in, 0);
      fdV[f] = make_field_desc(in, 1);
      for (int a = 0; a < 3; ++a) {
        idv[f].p[a] = in.p[a];
        idv[f].q[a] = in.q[a];
        idv[f].Ku[a] = fdU[f].K[a];
        kq[3 * f + a] = -in.q[a];
        kp[3 * f + a] = in.p[a];
      }
      idv[f].s = in.s;
      idv[f].r = in.r;
      idv[f].out = idx[f];
      idv[f].full = full ? 1 : 0;
      if (in.flags & SWF_WANT_SPECTRUM) any_spec = true;
    }
    const size_t state = (size_t)F * 4 * g.N;
    void *psiU, *specU, *uq, *normU, *pid;
    if ((s = ws_get(ctx, "solve.psiU", state * elem, &psiU)) != SWF_OK) return s;
    if ((s = ws_get(ctx, "solve.specU", state * 16, &specU)) != SWF_OK) return s;
    if ((s = ws_get(ctx, "solve.uq", (size_t)F * 64, &uq)) != SWF_OK) return s;
    if ((s = ws_get(ctx, "solve.normU", (size_t)F * 8, &normU)) != SWF_OK) return s;
    if ((s = ws_get(ctx, "solve.inst", sizeof(InstDev) * F, &pid)) != SWF_OK) return s;
    if (pre != premarched.end()) {
      psiU = pre->second;  // U fields, then (full) V fields
    } else if ((s = march_fields(ctx, g, i0.grid.t_in, i0.grid.t_out, i0.grid.n_steps, F, fdU.data(), prec, psiU, st,
                                 kv.first.adaptive)) != SWF_OK) {
      return s;
    }
    if ((s = transform_at(ctx, g, F, prec, psiU, kq.data(), (double2*)uq, st)) != SWF_OK) return s;
    if ((s = field_norms(ctx, g, F, prec, psiU, (double*)normU, st)) != SWF_OK) return s;
    if (any_spec || full)
      if ((s = transform_fields(ctx, g, F, prec, psiU, (double2*)specU, st)) != SWF_OK) return s;
    if (any_spec && spectrum_dev) {
      void* prob;
      if ((s = ws_get(ctx, "solve.prob", (size_t)F * 2 * g.N * 8, &prob)) != SWF_OK) return s;
      if ((s = c_spectrum(ctx, g, F, fdU.data(), i0.grid.t_in, (const double2*)specU, nullptr, (double*)prob, st)) != SWF_OK)
        return s;
      for (int f = 0; f < F; ++f) {
        if (!(inst[idx[f]].flags & SWF_WANT_SPECTRUM)) continue;
        cudaError_t e = cudaMemcpyAsync(spectrum_dev + spec_off[idx[f]], (double*)prob + (size_t)f * 2 * g.N,
                                        (size_t)2 * g.N * 8, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_status(e, "copy spectrum");
      }
    }
    void *psiV = nullptr, *specV = nullptr, *vp = nullptr, *normV = nullptr;
    if (full) {
      if ((s = ws_get(ctx, "solve.specV", state * 16, &specV)) != SWF_OK) return s;
      if ((s = ws_get(ctx, "solve.vp", (size_t)F * 64, &vp)) != SWF_OK) return s;
      if ((s = ws_get(ctx, "solve.normV", (size_t)F * 8, &normV)) != SWF_OK) return s;
      if (pre != premarched.end()) {
        psiV = (unsigned char*)pre->second + state * elem;
      } else {
        if ((s = ws_get(ctx, "solve.psiV", state * elem, &psiV)) != SWF_OK) return s;
        if ((s = march_fields(ctx, g, i0.grid.t_in, i0.grid.t_out, i0.grid.n_steps, F, fdV.data(), prec, psiV, st,
                              kv.first.adaptive)) != SWF_OK)
          return s;
      }
      if ((s = transform_fields(ctx, g, F, prec, psiV, (double2*)specV, st)) != SWF_OK) return s;
      if ((s = transform_at(ctx, g, F, prec, psiV, kp.data(), (double2*)vp, st)) != SWF_OK) return s;
      if ((s = field_norms(ctx, g, F, prec, psiV, (double*)normV, st)) != SWF_OK) return s;
    }
    cudaError_t e = cudaMemcpyAsync(pid, idv.data(), sizeof(InstDev) * F, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_status(e, "upload instance table");
    ProfScope ps(ctx, "finalize", st);
    k_finalize<<<F, 256, 0, st>>>((const InstDev*)pid, g, i0.grid.t_in, (const cpx<double>*)specU,
                                  (const cpx<double>*)specV, (const cpx<double>*)uq, (const cpx<double>*)vp,
                                  (const double*)normU, (const double*)normV, results_dev);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_status(e, "finalize kernel");
    // the host-side tables above must outlive the asynchronous uploads
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e, "group synchronisation");
  }
  return SWF_OK;
}

// The photon momentum must be a grid mode along non-trivial axes (the V mode of the past terms is
// the U mode minus k); along trivial axes momentum is conserved (p + q = k); k0 > 0.
static swf_status check_bw_photon(const swf_instance& in, const double* k, const std::string& pre) {
  for (int a = 0; a < 3; ++a) {
    if (in.grid.n[a] > 1) {
      const double m = k[a] * in.grid.L[a] / 6.283185307179586476925286766559;
      if (std::fabs(m - std::round(m)) > 1e-6) {
        set_error(pre + "the photon momentum must be a grid mode");
        return SWF_EINVAL;
      }
    } else if (std::fabs(in.p[a] + in.q[a] - k[a]) > 1e-9) {
      set_error(pre + "p + q must equal k along trivial axes");
      return SWF_EINVAL;
    }
  }
  if (!(std::sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]) > 0.0)) {
    set_error(pre + "the photon momentum must be non-zero");
    return SWF_EINVAL;
  }
  return SWF_OK;
}

static void photon_shift(const swf_instance& in, const double* k, int shift[3]) {
  for (int a = 0; a < 3; ++a)
    shift[a] = in.grid.n[a] > 1 ? (int)std::lround(k[a] * in.grid.L[a] / 6.283185307179586476925286766559) : 0;
}

// Marches, in multi-grid marches, every fixed-step Breit-Wheeler group of the past/finite form
// (Eq. 17) that shares its time grid and non-trivial axes with another such group (at most eight
// groups per march).  premarched[group] = (psi(t_in) [2G][4][N], the integrals of Eq. 17 [G][3]).
static swf_status premarch_bw(swf_ctx* ctx, const swf_instance* inst, const std::map<GroupKey, std::vector<int>>& groups,
                              swf_precision prec, std::map<const GroupKey*, std::pair<void*, void*>>& premarched,
                              cudaStream_t st) {
  if (!ctx->multi_grid) return SWF_OK;
  const size_t elem = prec == SWF_C64 ? 8 : 16;
  std::map<MultiKey, std::vector<const GroupKey*>> sets;
  for (auto& kv : groups) {
    if (kv.first.adaptive || kv.first.full) continue;
    const swf_instance& i0 = inst[kv.second[0]];
    sets[MultiKey{i0.grid.t_in, i0.grid.t_out, i0.grid.n_steps, i0.grid.n[1] > 1, i0.grid.n[2] > 1}].push_back(
        &kv.first);
  }
  swf_status s;
  int buf = 0;
  for (auto& kv : sets) {
    const std::vector<const GroupKey*>& list = kv.second;
    for (size_t b = 0; b + 1 < list.size(); b += 8) {
      const size_t e = std::min(list.size(), b + 8);
      double sites = 0.0;  // U and V of every instance
      for (size_t i = b; i < e; ++i)
        sites += 2.0 * groups.at(*list[i]).size() * make_grid(inst[groups.at(*list[i])[0]].grid).N;
      if (ctx->multi_grid == 1 && sites >= kMultiAutoSites) continue;
      std::vector<std::vector<FieldDesc>> fds(e - b);
      std::vector<std::vector<double>> photons(e - b);
      std::vector<MultiGroup> mg;
      for (size_t i = b; i < e; ++i) {
        const std::vector<int>& idx = groups.at(*list[i]);
        const int G = (int)idx.size();
        const GridDesc g = make_grid(inst[idx[0]].grid);
        std::vector<FieldDesc>& fd = fds[i - b];
        std::vector<double>& ph = photons[i - b];
        fd.resize(2 * G);
        ph.resize(6 * G);
        for (int f = 0; f < G; ++f) {
          const swf_instance& in = inst[idx[f]];
          fd[2 * f] = make_field_desc(in, 0);
          fd[2 * f + 1] = make_field_desc(in, 1);
          for (int a = 0; a < 3; ++a) {
            ph[6 * f + a] = in.k[a];
            ph[6 * f + 3 + a] = in.eps[a];
          }
        }
        void *psi = nullptr, *macc = nullptr;
        const std::string tag = "bwsolve.multi" + std::to_string(buf++);
        if ((s = ws_get(ctx, tag + ".psi", (size_t)2 * G * 4 * g.N * elem, &psi)) != SWF_OK) return s;
        if ((s = ws_get(ctx, tag + ".macc", (size_t)G * 9 * 16, &macc)) != SWF_OK) return s;
        mg.push_back(MultiGroup{g, 2 * G, fd.data(), psi, ph.data(), (double2*)macc});
        premarched[list[i]] = {psi, macc};
      }
      s = march_multi(ctx, mg, kv.first.t_in, kv.first.t_out, kv.first.n_steps, prec, 1, st);
      if (s == SWF_EUNSUPPORTED) {  // not a form the grouped launch takes: these groups march alone
        for (size_t i = b; i < e; ++i) premarched.erase(list[i]);
        continue;
      }
      if (s != SWF_OK) return s;
    }
  }
  return SWF_OK;
}

// Breit-Wheeler (Sec. IV): U and V marched together per instance, then past terms and totals.
static swf_status solve_bw(swf_ctx* ctx, int n_inst, const swf_instance* inst, swf_precision prec,
                           swf_result* results_dev, cudaStream_t st) {
  std::map<GroupKey, std::vector<int>> groups;
  for (int i = 0; i < n_inst; ++i) {
    const swf_instance& in = inst[i];
    GroupKey k;
    for (int a = 0; a < 3; ++a) { k.n[a] = in.grid.n[a]; k.L[a] = in.grid.n[a] > 1 ? in.grid.L[a] : 0.0; }
    k.t_in = in.grid.t_in;
    k.t_out = in.grid.t_out;
    k.n_steps = in.grid.n_steps;
    k.full = (in.flags & SWF_BW_PARTIAL) ? 1 : 0;  // the integrand form (Eq. 17 + past, or Eqs. 30-33)
    k.adaptive = (in.flags & SWF_ADAPTIVE) ? 1 : 0;
    groups[k].push_back(i);
    if ((in.flags & SWF_ADAPTIVE) && (in.flags & SWF_BW_PARTIAL)) {
      set_error("instance " + std::to_string(i) +
                ": the partial-integration form marches at fixed steps (step-size control is for the past/finite split)");
      return SWF_EUNSUPPORTED;
    }
    swf_status c = check_bw_photon(in, in.k, "instance " + std::to_string(i) + ": ");
    if (c != SWF_OK) return c;
  }
  const size_t elem = prec == SWF_C64 ? 8 : 16;
  swf_status s;
  // fixed-step groups of the past/finite form that share a time grid and their non-trivial axes:
  // marched together (U, V and the integrals of Eq. 17) in multi-grid marches
  std::map<const GroupKey*, std::pair<void*, void*>> premarched;
  if ((s = premarch_bw(ctx, inst, groups, prec, premarched, st)) != SWF_OK) return s;
  for (auto& kv : groups) {
    const std::vector<int>& idx = kv.second;
    const int G = (int)idx.size();
    const int form = kv.first.full ? 2 : 1;
    auto pre = premarched.find(&kv.first);
    const swf_instance& i0 = inst[idx[0]];
    const GridDesc g = make_grid(i0.grid);
    std::vector<FieldDesc> fd(2 * G);
    std::vector<double> photon(6 * G), kat(6 * G);
    std::vector<unsigned char> bw(bw_inst_size() * G);
    for (int f = 0; f < G; ++f) {
      const swf_instance& in = inst[idx[f]];
      fd[2 * f] = make_field_desc(in, 0);
      fd[2 * f + 1] = make_field_desc(in, 1);
      int shift[3];
      photon_shift(in, in.k, shift);
      for (int a = 0; a < 3; ++a) {
        photon[6 * f + a] = in.k[a];
        photon[6 * f + 3 + a] = in.eps[a];
        kat[6 * f + a] = in.k[a] - in.q[a];      // U~ at k - q
        kat[6 * f + 3 + a] = in.p[a] - in.k[a];  // V~ at p - k
      }
      bw_fill_inst(bw.data() + bw_inst_size() * f, in, idx[f], fd[2 * f], fd[2 * f + 1], shift, f);
    }
    const size_t state = (size_t)2 * G * 4 * g.N;
    void *psi, *spec, *tat, *macc, *norms;
    if ((s = ws_get(ctx, "bwsolve.spec", state * 16, &spec)) != SWF_OK) return s;
    if ((s = ws_get(ctx, "bwsolve.tat", (size_t)2 * G * 64, &tat)) != SWF_OK) return s;
    if ((s = ws_get(ctx, "bwsolve.norms", (size_t)2 * G * 8, &norms)) != SWF_OK) return s;
    if (pre != premarched.end()) {
      psi = pre->second.first;
      macc = pre->second.second;
    } else {
      if ((s = ws_get(ctx, "bwsolve.psi", state * elem, &psi)) != SWF_OK) return s;
      if ((s = ws_get(ctx, "bwsolve.macc", (size_t)G * 9 * 16, &macc)) != SWF_OK) return s;
    }
    // kat holds, per wave, the momentum of its direct transform (U~ at k - q, V~ at p - k)
    if (pre != premarched.end()) {
      // marched with the other groups of its time grid
    } else if (kv.first.adaptive) {
      // first step (t_in - t_out)/n_steps, at most 100 n_steps + 100 attempts (as for Schwinger marches)
      const double h0 = (i0.grid.t_in - i0.grid.t_out) / i0.grid.n_steps;
      if ((s = march_bw_adaptive(ctx, g, i0.grid.t_in, i0.grid.t_out, h0, 100 * i0.grid.n_steps + 100, G, fd.data(),
                                 photon.data(), prec, psi, (double2*)macc, st)) != SWF_OK)
        return s;
    } else if ((s = march_bw(ctx, g, i0.grid.t_in, i0.grid.t_out, i0.grid.n_steps, G, fd.data(), photon.data(), prec,
                             psi, (double2*)macc, st, form, kat.data())) != SWF_OK) {
      return s;
    }
    if (form == 2) {
      if ((s = field_norms(ctx, g, 2 * G, prec, psi, (double*)norms, st)) != SWF_OK) return s;
      if ((s = bw_finalize_partial(ctx, g, G, bw.data(), (const double2*)macc, (const double*)norms, results_dev,
                                   st)) != SWF_OK)
        return s;
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return cuda_status(e, "Breit-Wheeler group");
      continue;
    }
    if ((s = transform_fields(ctx, g, 2 * G, prec, psi, (double2*)spec, st)) != SWF_OK) return s;
    if ((s = transform_at(ctx, g, 2 * G, prec, psi, kat.data(), (double2*)tat, st)) != SWF_OK) return s;
    if ((s = field_norms(ctx, g, 2 * G, prec, psi, (double*)norms, st)) != SWF_OK) return s;
    if ((s = bw_finalize(ctx, g, G, bw.data(), i0.grid.t_in, (const double2*)spec, (const double2*)tat,
                         (const double2*)macc, (const double*)norms, results_dev, st)) != SWF_OK)
      return s;
    cudaError_t e = cudaStreamSynchronize(st);  // host tables above are temporaries
    if (e != cudaSuccess) return cuda_status(e, "Breit-Wheeler group");
  }
  return SWF_OK;
}

// Photon scan (Sec. IV): one march of U and V, the amplitudes of n photons (k_j, eps_j), and their
// weighted sum.  Host outputs; synchronous.
static swf_status bw_photon_scan(swf_ctx* ctx, const swf_instance& in, int n, const double* k, const double* eps,
                                 const double* weights, swf_precision prec, double* amp_out, double* packet_out) {
  cudaStream_t st = ctx->stream;
  const GridDesc g = make_grid(in.grid);
  const FieldDesc fd[2] = {make_field_desc(in, 0), make_field_desc(in, 1)};
  std::vector<double> photon(6 * (size_t)n), kat(6 * (size_t)n);
  std::vector<unsigned char> bw(bw_inst_size() * (size_t)n);
  for (int j = 0; j < n; ++j) {
    swf_instance ij = in;
    int shift[3];
    for (int a = 0; a < 3; ++a) {
      ij.k[a] = k[3 * j + a];
      ij.eps[a] = eps[3 * j + a];
      photon[6 * j + a] = ij.k[a];
      photon[6 * j + 3 + a] = ij.eps[a];
      kat[6 * j + a] = ij.k[a] - in.q[a];      // U~ at k_j - q
      kat[6 * j + 3 + a] = in.p[a] - ij.k[a];  // V~ at p - k_j
    }
    photon_shift(in, ij.k, shift);
    bw_fill_inst(bw.data() + bw_inst_size() * j, ij, j, fd[0], fd[1], shift, 0);
  }
  const size_t elem = prec == SWF_C64 ? 8 : 16;
  void *psi, *spec, *tat, *macc, *norms, *res, *pk;
  swf_status s;
  if ((s = ws_get(ctx, "bwscan.psi", (size_t)2 * 4 * g.N * elem, &psi)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bwscan.spec", (size_t)2 * 4 * g.N * 16, &spec)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bwscan.tat", (size_t)n * 8 * 16, &tat)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bwscan.macc", (size_t)n * 3 * 16, &macc)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bwscan.norms", 2 * 8, &norms)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bwscan.results", sizeof(swf_result) * (size_t)n, &res)) != SWF_OK) return s;
  if ((s = ws_get(ctx, "bwscan.packet", 4 * 16, &pk)) != SWF_OK) return s;
  if ((s = march_bw(ctx, g, in.grid.t_in, in.grid.t_out, in.grid.n_steps, 1, fd, photon.data(), prec, psi,
                    (double2*)macc, st, 1, nullptr, n)) != SWF_OK)
    return s;
  if ((s = transform_fields(ctx, g, 2, prec, psi, (double2*)spec, st)) != SWF_OK) return s;
  for (int j = 0; j < n; ++j)
    if ((s = transform_at(ctx, g, 2, prec, psi, kat.data() + 6 * j, (double2*)tat + 8 * j, st)) != SWF_OK) return s;
  if ((s = field_norms(ctx, g, 2, prec, psi, (double*)norms, st)) != SWF_OK) return s;
  if ((s = bw_finalize(ctx, g, n, bw.data(), in.grid.t_in, (const double2*)spec, (const double2*)tat,
                       (const double2*)macc, (const double*)norms, (swf_result*)res, st)) != SWF_OK)
    return s;
  if (packet_out && (s = bw_packet(ctx, n, (const swf_result*)res, weights, (double2*)pk, st)) != SWF_OK) return s;
  std::vector<swf_result> host(n);
  cudaError_t e = cudaMemcpyAsync(host.data(), res, sizeof(swf_result) * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_status(e, "copy photon-scan results");
  if (packet_out && (e = cudaMemcpyAsync(packet_out, pk, 4 * 16, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_status(e, "copy packet amplitude");
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "photon scan");
  for (int j = 0; j < n; ++j)
    for (int c = 0; c < 8; ++c) amp_out[8 * j + c] = host[j].amp[c];
  return SWF_OK;
}

static size_t spectrum_len(int n_inst, const swf_instance* inst, swf_process process) {
  size_t n = 0;
  if (process != SWF_SCHWINGER) return 0;
  for (int i = 0; i < n_inst; ++i)
    if (inst[i].flags & SWF_WANT_SPECTRUM) n += (size_t)2 * inst[i].grid.n[0] * inst[i].grid.n[1] * inst[i].grid.n[2];
  return n;
}

}  // namespace swf

using namespace swf;

extern "C" {

const char* swf_last_error(void) { return g_err.c_str(); }

swf_status swf_create(swf_ctx** ctx, int device) {
  if (!ctx) { set_error("ctx is NULL"); return SWF_EINVAL; }
  *ctx = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    set_error("CUDA device " + std::to_string(device) + " not available");
    return SWF_ECUDA;
  }
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_status(e, "cudaSetDevice");
  swf_ctx* c = new swf_ctx();
  c->device = device;
  e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete c;
    return cuda_status(e, "cudaStreamCreate");
  }
  *ctx = c;
  return SWF_OK;
}

swf_status swf_destroy(swf_ctx* ctx) {
  if (!ctx) return SWF_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->ws.bufs) cudaFree(kv.second.first);
  for (auto& kv : ctx->tw.tables) cudaFree(kv.second);
  for (auto ev : ctx->prof.pool) cudaEventDestroy(ev);
  if (ctx->aux) {
    cudaStreamSynchronize(ctx->aux);
    for (auto ev : ctx->aux_ev)
      if (ev) cudaEventDestroy(ev);
    cudaStreamDestroy(ctx->aux);
  }
  cudaStreamDestroy(ctx->stream);
  delete ctx;
  return SWF_OK;
}

swf_status swf_profile_enable(swf_ctx* ctx, int on) {
  if (!ctx) { set_error("ctx is NULL"); return SWF_EINVAL; }
  ctx->prof.on = on != 0;
  return SWF_OK;
}

swf_status swf_profile_read(swf_ctx* ctx, int max_entries, char* names, double* total_ms, long long* launches,
                            int* n_entries, long long* total_launches) {
  if (!ctx || max_entries < 0 || (max_entries > 0 && (!names || !total_ms || !launches)) || !n_entries) {
    set_error("swf_profile_read: invalid arguments");
    return SWF_EINVAL;
  }
  Profiler& P = ctx->prof;
  for (auto& m : P.marks) {
    cudaEvent_t a = P.pool[m.second], b = P.pool[m.second + 1];
    cudaError_t e = cudaEventSynchronize(b);
    if (e != cudaSuccess) return cuda_status(e, "cudaEventSynchronize");
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess) return cuda_status(e, "cudaEventElapsedTime");
    auto& slot = P.acc[P.families[m.first]];
    slot.first += ms;
    slot.second += 1;
  }
  P.marks.clear();
  P.used = 0;
  int n = 0;
  for (auto& kv : P.acc) {
    if (n >= max_entries) break;
    std::snprintf(names + 32 * n, 32, "%s", kv.first.c_str());
    total_ms[n] = kv.second.first;
    launches[n] = kv.second.second;
    ++n;
  }
  *n_entries = n;
  if (total_launches) *total_launches = P.launches;
  P.acc.clear();
  P.launches = 0;
  return SWF_OK;
}

swf_status swf_set_march_path(swf_ctx* ctx, int path) {
  if (!ctx || path < 0 || path > 5) { set_error("swf_set_march_path: ctx NULL or path not in 0..5"); return SWF_EINVAL; }
  ctx->use_fused = path != 1;
  ctx->sm_split = path == 0;
  ctx->fused_variant = path == 3 ? 2 : path == 4 ? 1 : path == 5 ? 3 : kDefaultFusedVariant;
  return SWF_OK;
}

swf_status swf_fused_status(swf_ctx* ctx, int* status) {
  if (!ctx || !status) { set_error("swf_fused_status: NULL argument"); return SWF_EINVAL; }
  *status = 0;
  if (!ctx->fused_status_dev) return SWF_OK;
  // the march may have run on a caller's stream (swf_march_dev, solve_swf_dev): wait for the device
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(status, ctx->fused_status_dev, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e, "read the fused kernel's status");
  return SWF_OK;
}

swf_status swf_set_fused_drop(swf_ctx* ctx, int on) {
  if (!ctx) { set_error("swf_set_fused_drop: ctx is NULL"); return SWF_EINVAL; }
  ctx->fused_drop = on ? 1 : 0;
  return SWF_OK;
}

swf_status swf_set_tolerances(swf_ctx* ctx, double rtol, double atol) {
  if (!ctx || !(rtol > 0.0) || !(atol > 0.0) || !std::isfinite(rtol) || !std::isfinite(atol)) {
    set_error("swf_set_tolerances: need ctx and positive finite rtol, atol");
    return SWF_EINVAL;
  }
  ctx->rtol = rtol;
  ctx->atol = atol;
  return SWF_OK;
}

swf_status swf_march_stats(swf_ctx* ctx, long long* accepted, long long* rejected) {
  if (!ctx || !accepted || !rejected) { set_error("swf_march_stats: NULL argument"); return SWF_EINVAL; }
  *accepted = ctx->last_accepted;
  *rejected = ctx->last_rejected;
  return SWF_OK;
}

swf_status swf_set_dedupe(swf_ctx* ctx, int on) {
  if (!ctx || (on != 0 && on != 1)) { set_error("swf_set_dedupe: ctx NULL or on not 0 or 1"); return SWF_EINVAL; }
  ctx->dedupe = on != 0;
  return SWF_OK;
}

swf_status swf_set_multi_grid(swf_ctx* ctx, int mode) {
  if (!ctx || mode < 0 || mode > 2) { set_error("swf_set_multi_grid: ctx NULL or mode not 0, 1 or 2"); return SWF_EINVAL; }
  ctx->multi_grid = mode;
  return SWF_OK;
}

swf_status swf_device_loop_marches(swf_ctx* ctx, long long* count) {
  if (!ctx || !count) { set_error("swf_device_loop_marches: NULL argument"); return SWF_EINVAL; }
  *count = ctx->device_loop_marches;
  return SWF_OK;
}

swf_status swf_fields_marched(swf_ctx* ctx, long long* count) {
  if (!ctx || !count) { set_error("swf_fields_marched: NULL argument"); return SWF_EINVAL; }
  *count = ctx->fields_marched;
  return SWF_OK;
}

swf_status swf_plan_split(int n_fields, int clusters, int sms, int* pass_fields) {
  if (!pass_fields || n_fields < 0 || clusters < 0 || sms < 0) {
    set_error("swf_plan_split: negative count or NULL pointer");
    return SWF_EINVAL;
  }
  *pass_fields = fused_split_count(n_fields, clusters, sms);
  return SWF_OK;
}

swf_status swf_fields_fused(swf_ctx* ctx, long long* count) {
  if (!ctx || !count) { set_error("swf_fields_fused: NULL argument"); return SWF_EINVAL; }
  *count = ctx->fields_fused;
  return SWF_OK;
}

swf_status swf_set_autotune(swf_ctx* ctx, int on) {
  if (!ctx || (on != 0 && on != 1)) { set_error("swf_set_autotune: ctx NULL or on not 0 or 1"); return SWF_EINVAL; }
  ctx->tune.on = on != 0;
  return SWF_OK;
}

swf_status swf_set_workspace_limit(swf_ctx* ctx, size_t bytes) {
  if (!ctx) { set_error("ctx is NULL"); return SWF_EINVAL; }
  ctx->ws.limit = bytes;
  return SWF_OK;
}

swf_status solve_swf_dev(swf_ctx* ctx, int n_inst, const swf_instance* inst, swf_process process,
                         swf_precision prec, swf_result* results_dev, double* spectrum_dev, void* stream) {
  if (!ctx) { set_error("ctx is NULL"); return SWF_EINVAL; }
  swf_status s = validate(n_inst, inst, process, prec);
  if (s != SWF_OK) return s;
  if (n_inst > 0 && !results_dev) { set_error("results pointer is NULL"); return SWF_EINVAL; }
  if (n_inst == 0) return SWF_OK;
  cudaSetDevice(ctx->device);
  cudaStream_t st = pick_stream(ctx, stream);
  if (process == SWF_SCHWINGER) return solve_schwinger(ctx, n_inst, inst, prec, results_dev, spectrum_dev, st);
  return solve_bw(ctx, n_inst, inst, prec, results_dev, st);
}

swf_status solve_swf(swf_ctx* ctx, int n_inst, const swf_instance* inst, swf_process process,
                     swf_precision prec, swf_result* results, double* spectrum) {
  if (!ctx) { set_error("ctx is NULL"); return SWF_EINVAL; }
  swf_status s = validate(n_inst, inst, process, prec);
  if (s != SWF_OK) return s;
  if (n_inst > 0 && !results) { set_error("results pointer is NULL"); return SWF_EINVAL; }
  if (n_inst == 0) return SWF_OK;
  cudaSetDevice(ctx->device);
  void *rd = nullptr, *sd = nullptr;
  if ((s = ws_get(ctx, "host.results", sizeof(swf_result) * n_inst, &rd)) != SWF_OK) return s;
  const size_t slen = spectrum ? spectrum_len(n_inst, inst, process) : 0;
  if (slen && (s = ws_get(ctx, "host.spectrum", slen * 8, &sd)) != SWF_OK) return s;
  s = solve_swf_dev(ctx, n_inst, inst, process, prec, (swf_result*)rd, slen ? (double*)sd : nullptr, ctx->stream);
  if (s != SWF_OK) return s;
  cudaError_t e = cudaMemcpyAsync(results, rd, sizeof(swf_result) * n_inst, cudaMemcpyDeviceToHost, ctx->stream);
  if (e != cudaSuccess) return cuda_status(e, "copy results");
  if (slen) {
    e = cudaMemcpyAsync(spectrum, sd, slen * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return cuda_status(e, "copy spectrum");
  }
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_status(e, "stream synchronisation");
  return SWF_OK;
}

swf_status swf_bw_photons(swf_ctx* ctx, const swf_instance* inst, int n_photons, const double* k, const double* eps,
                          const double* weights, swf_precision prec, double* amp_out, double* packet_out) {
  if (!ctx) { set_error("ctx is NULL"); return SWF_EINVAL; }
  swf_status s = validate(1, inst, SWF_BREIT_WHEELER, prec);
  if (s != SWF_OK) return s;
  if (n_photons < 1 || !k || !eps || !amp_out) {
    set_error("need n_photons >= 1 and the k, eps and amp_out pointers");
    return SWF_EINVAL;
  }
  if (packet_out && !weights) { set_error("packet_out needs weights"); return SWF_EINVAL; }
  if (inst->flags & (SWF_ADAPTIVE | SWF_BW_PARTIAL)) {
    set_error("photon scans march at fixed steps with the past/finite split of the amplitude");
    return SWF_EUNSUPPORTED;
  }
  for (int j = 0; j < n_photons; ++j) {
    const std::string pre = "photon " + std::to_string(j) + ": ";
    if (!finite3(k + 3 * j) || !finite3(eps + 3 * j) ||
        (weights && !(std::isfinite(weights[2 * j]) && std::isfinite(weights[2 * j + 1])))) {
      set_error(pre + "momentum, polarisation and weight must be finite");
      return SWF_EINVAL;
    }
    if ((s = check_bw_photon(*inst, k + 3 * j, pre)) != SWF_OK) return s;
  }
  cudaSetDevice(ctx->device);
  return bw_photon_scan(ctx, *inst, n_photons, k, eps, weights, prec, amp_out, packet_out);
}

swf_status swf_march_dev(swf_ctx* ctx, int n_inst, const swf_instance* inst, int bg, swf_precision prec,
                         void* psi_out_dev, void* stream) {
  if (!ctx) { set_error("ctx is NULL"); return SWF_EINVAL; }
  swf_status s = validate(n_inst, inst, SWF_SCHWINGER, prec);
  if (s != SWF_OK) return s;
  if (bg != 0 && bg != 1) { set_error("bg must be 0 (U) or 1 (V)"); return SWF_EINVAL; }
  if (n_inst == 0) return SWF_OK;
  if (!psi_out_dev) { set_error("psi_out_dev is NULL"); return SWF_EINVAL; }
  for (int i = 1; i < n_inst; ++i) {
    const swf_grid &a = inst[0].grid, &b = inst[i].grid;
    if (std::memcmp(a.n, b.n, sizeof a.n) || a.n_steps != b.n_steps || a.t_in != b.t_in || a.t_out != b.t_out ||
        std::memcmp(a.L, b.L, sizeof a.L) || ((inst[0].flags ^ inst[i].flags) & SWF_ADAPTIVE)) {
      set_error("swf_march_dev: all instances must share the grid, time window and step control");
      return SWF_EINVAL;
    }
  }
  cudaSetDevice(ctx->device);
  cudaStream_t st = pick_stream(ctx, stream);
  std::vector<FieldDesc> fd(n_inst);
  for (int i = 0; i < n_inst; ++i) fd[i] = make_field_desc(inst[i], bg);
  const GridDesc g = make_grid(inst[0].grid);
  s = march_fields(ctx, g, inst[0].grid.t_in, inst[0].grid.t_out, inst[0].grid.n_steps, n_inst, fd.data(), prec,
                   psi_out_dev, st, (inst[0].flags & SWF_ADAPTIVE) ? 1 : 0);
  if (s != SWF_OK) return s;
  cudaError_t e = cudaStreamSynchronize(st);  // fd lives on this stack frame
  if (e != cudaSuccess) return cuda_status(e, "march synchronisation");
  return SWF_OK;
}

swf_status swf_rhs_dev(swf_ctx* ctx, const swf_instance* inst, int bg, swf_precision prec, double t,
                       const void* psi_dev, void* out_dev, void* stream) {
  if (!ctx) { set_error("ctx is NULL"); return SWF_EINVAL; }
  swf_status s = validate(1, inst, SWF_SCHWINGER, prec);
  if (s != SWF_OK) return s;
  if (bg != 0 && bg != 1) { set_error("bg must be 0 (U) or 1 (V)"); return SWF_EINVAL; }
  if (!psi_dev || !out_dev || psi_dev == out_dev) { set_error("psi_dev/out_dev must be distinct device pointers"); return SWF_EINVAL; }
  if (!std::isfinite(t)) { set_error("t must be finite"); return SWF_EINVAL; }
  cudaSetDevice(ctx->device);
  cudaStream_t st = pick_stream(ctx, stream);
  const FieldDesc fd = make_field_desc(*inst, bg);
  s = rhs_eval(ctx, make_grid(inst->grid), fd, prec, t, psi_dev, out_dev, st);
  if (s != SWF_OK) return s;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "rhs synchronisation");
  return SWF_OK;
}

swf_status swf_spectrum_dev(swf_ctx* ctx, int n_inst, const swf_instance* inst, swf_precision prec,
                            const void* psi_dev, double* c_out_dev, double* prob_out_dev, void* stream) {
  if (!ctx) { set_error("ctx is NULL"); return SWF_EINVAL; }
  swf_status s = validate(n_inst, inst, SWF_SCHWINGER, prec);
  if (s != SWF_OK) return s;
  if (n_inst == 0) return SWF_OK;
  if (!psi_dev || (!c_out_dev && !prob_out_dev)) { set_error("need psi_dev and an output"); return SWF_EINVAL; }
  for (int i = 1; i < n_inst; ++i)
    if (std::memcmp(inst[0].grid.n, inst[i].grid.n, sizeof inst[0].grid.n) ||
        std::memcmp(inst[0].grid.L, inst[i].grid.L, sizeof inst[0].grid.L)) {
      set_error("swf_spectrum_dev: all instances must share the grid");
      return SWF_EINVAL;
    }
  cudaSetDevice(ctx->device);
  cudaStream_t st = pick_stream(ctx, stream);
  const GridDesc g = make_grid(inst[0].grid);
  std::vector<FieldDesc> fd(n_inst);
  for (int i = 0; i < n_inst; ++i) fd[i] = make_field_desc(inst[i], 0);
  void* spec;
  if ((s = ws_get(ctx, "spec.tmp", (size_t)n_inst * 4 * g.N * 16, &spec)) != SWF_OK) return s;
  if ((s = transform_fields(ctx, g, n_inst, prec, psi_dev, (double2*)spec, st)) != SWF_OK) return s;
  if ((s = c_spectrum(ctx, g, n_inst, fd.data(), inst[0].grid.t_in, (const double2*)spec, (double2*)c_out_dev,
                      prob_out_dev, st)) != SWF_OK)
    return s;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e, "spectrum synchronisation");
  return SWF_OK;
}

}  // extern "C"
