// Internal declarations shared by the SWF library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/swf.h"
#include "swf_common.cuh"

namespace swf {

// One marched 4-spinor field: the background plane wave and the gauge field it sees.
struct FieldDesc {
  int kind;        // swf_field_kind
  int acomp;       // index mu of the one non-zero A_mu (-1 for the zero field)
  double prm[8];
  double w[8];     // background spinor u_s(p) or v_r(q): (re, im) x 4
  double e0;       // background energy p0 (or q0)
  double tsign;    // time phase exp(i tsign e0 t): -1 for U, +1 for V
  double K[3];     // momentum carried along trivial axes
  double pmom[3];  // spatial phase exp(i pmom.x): p for U, -q for V
};

// Grid of one group of instances (all instances of a launch share it).
struct GridDesc {
  int n[3];
  double L[3];
  int N;        // n0 n1 n2
  double dx[3]; // cell widths (1 on trivial axes)
  double x0[3]; // first coordinate (-L/2, or 0 on trivial axes)
};

GridDesc make_grid(const swf_grid& g);

// Spinors of Eq. A44 in the Dirac representation, FP64, host and device:
// u_s(p) = (1 + p-slash) R_s / sqrt(2 p0 (p0 - p^x)), v_s(p) = (1 - p-slash) R_s / (same),
// with p-slash = [[p0, -sigma.p], [sigma.p, -p0]], R_+ = (1,1,1,1)/2, R_- = (1,-1,-1,1)/2.
// out = (re, im) of the four components.
__host__ __device__ inline void spinor_uv(const double p[3], int s, bool is_v, double out[8]) {
  const double p0 = sqrt(1.0 + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  const double nrm = 1.0 / sqrt(2.0 * p0 * (p0 - p[0]));
  const double ru0 = 0.5, ru1 = s > 0 ? 0.5 : -0.5;  // upper half of R_s
  const double rl0 = s > 0 ? 0.5 : -0.5, rl1 = 0.5;  // lower half of R_s
  // sigma.p applied to a real 2-vector (a, b): (pz a + px b - i py b, px a - pz b + i py a)
  const double spl_re0 = p[2] * rl0 + p[0] * rl1, spl_im0 = -p[1] * rl1;
  const double spl_re1 = p[0] * rl0 - p[2] * rl1, spl_im1 = p[1] * rl0;
  const double spu_re0 = p[2] * ru0 + p[0] * ru1, spu_im0 = -p[1] * ru1;
  const double spu_re1 = p[0] * ru0 - p[2] * ru1, spu_im1 = p[1] * ru0;
  const double sg = is_v ? -1.0 : 1.0;  // u: 1 + p-slash, v: 1 - p-slash
  // upper = (1 + sg p0) R_u - sg sigma.p R_l ; lower = sg sigma.p R_u + (1 - sg p0) R_l
  out[0] = ((1.0 + sg * p0) * ru0 - sg * spl_re0) * nrm;
  out[1] = (-sg * spl_im0) * nrm;
  out[2] = ((1.0 + sg * p0) * ru1 - sg * spl_re1) * nrm;
  out[3] = (-sg * spl_im1) * nrm;
  out[4] = (sg * spu_re0 + (1.0 - sg * p0) * rl0) * nrm;
  out[5] = (sg * spu_im0) * nrm;
  out[6] = (sg * spu_re1 + (1.0 - sg * p0) * rl1) * nrm;
  out[7] = (sg * spu_im1) * nrm;
}
__host__ __device__ inline double energy3(const double p[3]) { return sqrt(1.0 + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]); }
__host__ __device__ inline double mode_kappa(int j, int n, double L) {
  if (n <= 1) return 0.0;
  int jp = (j < (n + 1) / 2) ? j : j - n;
  return 6.283185307179586476925286766559 * (double)jp / L;
}

FieldDesc make_field_desc(const swf_instance& in, int bg);

// Builds the radix plan (radices 4, 2, 3, 5) of a length; false if n has another factor.
bool make_radix_plan(int n, RadixPlan* pl);

// Index of the current device for per-device set-up flags (kernel attributes are per device).
inline int dev_slot() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess || d < 0 || d >= 64) d = 0;
  return d;
}

// Device workspace: a growable pool of named buffers owned by the context.
struct Workspace {
  std::map<std::string, std::pair<void*, size_t>> bufs;
  size_t total = 0;
  size_t limit = 0;  // 0 = no cap
};

struct TwiddleCache {
  std::map<std::pair<int, int>, void*> tables;  // (n, is_double) -> device table
};

}  // namespace swf

namespace swf {
// Per-context kernel timing: event pairs recorded around launches, reduced on read.
struct Profiler {
  bool on = false;
  long long launches = 0;                                 // every launch, timed or not
  std::vector<cudaEvent_t> pool;                          // reusable events
  size_t used = 0;
  std::vector<std::pair<int, size_t>> marks;              // (family, first event index)
  std::vector<std::string> families;
  std::map<std::string, std::pair<double, long long>> acc;  // family -> (ms, launches)
};
}  // namespace swf

namespace swf {
// Launch shapes of the pass kernels chosen by timing, per shape key (see the march).
struct TuneCache {
  bool on = true;
  std::map<std::string, int> best;
};
}  // namespace swf

// Fused kernel of march paths 0 and 2: 1 = threads pull the transposes through distributed
// shared memory (k_fused), 3 = the bulk-copy engine pushes them while the threads compute (k_fused3).
constexpr int kDefaultFusedVariant = 3;
// CTAs per cluster of the fused kernels (one CTA per SM).
constexpr int kFusedClusterCtas = 16;

struct swf_ctx {
  int device;
  cudaStream_t stream;
  swf::Workspace ws;
  swf::TwiddleCache tw;
  swf::Profiler prof;
  swf::TuneCache tune;
  bool use_fused = true;  // route eligible marches to the fused cluster kernel
  bool dedupe = true;     // march fields that repeat another (the other spin) once
  bool use_graphs = true; // replay pass-kernel march steps from CUDA graphs
  double rtol = 1e-5, atol = 1e-10;  // step-size control (SWF_ADAPTIVE), the paper's tolerances
  long long last_accepted = 0, last_rejected = 0;  // steps of the last controlled march
  long long fields_marched = 0;  // fields actually marched since the context's creation
  long long fields_fused = 0;    // of those, fields marched by the fused cluster kernel
  int multi_grid = 1;            // grid groups sharing a time grid in one launch sequence: 0 never, 1 auto, 2 always
  long long multi_marches = 0;   // multi-grid marches run since the context's creation
  long long device_loop_marches = 0;  // step-size-controlled marches decided entirely on the device
  int fused_variant = kDefaultFusedVariant;  // 1: pulled transposes, 2: two CTAs per SM, 3: pushed
  int fused_drop = 0;                // diagnostic: the pushed-transpose kernel issues no copies
  int* fused_status_dev = nullptr;   // status word of the last fused launch (workspace)
  bool sm_split = true;   // automatic path: pass kernels on the SMs the fused clusters leave free
  cudaStream_t aux = nullptr;            // stream of that concurrent pass-kernel march (lazy)
  cudaEvent_t aux_ev[2] = {nullptr, nullptr};
};

namespace swf {

void set_error(const std::string& msg);
swf_status validate_instances(int n_inst, const swf_instance* inst, swf_precision prec);

// Kernel timing: call prof_begin before a launch and prof_end after it (same stream).
int prof_begin(swf_ctx* ctx, const char* family, cudaStream_t st);
void prof_end(swf_ctx* ctx, int mark, cudaStream_t st);
struct ProfScope {
  swf_ctx* ctx;
  int mark;
  cudaStream_t st;
  ProfScope(swf_ctx* c, const char* fam, cudaStream_t s) : ctx(c), mark(c ? prof_begin(c, fam, s) : -1), st(s) {}
  ~ProfScope() {
    if (ctx) prof_end(ctx, mark, st);
  }
};
swf_status cuda_status(cudaError_t e, const char* what);

// Returns a device buffer of at least `bytes` under `name` (grows, never shrinks).
swf_status ws_get(swf_ctx* ctx, const std::string& name, size_t bytes, void** ptr);
// Device table exp(-2 pi i m/n), m < n, in float2 (is_double = 0) or double2.
swf_status twiddles(swf_ctx* ctx, int n, int is_double, const void** ptr);

// ---- march (swf_march.cu)
// March n_f fields (all on grid g) from psi(t_out) = 0 to t_in; psi_out receives psi(t_in)
// in the march precision [F][4][N].  fd_host: n_f descriptors.
swf_status march_fields(swf_ctx* ctx, const GridDesc& g, double t_in, double t_out, int n_steps,
                        int n_f, const FieldDesc* fd_host, swf_precision prec, void* psi_out,
                        cudaStream_t st, int adaptive = 0);
// Step-size-controlled march (first step h0, at most max_attempts attempts; tolerances from ctx)
swf_status march_adaptive(swf_ctx* ctx, const GridDesc& g, double t_in, double t_out, double h0, int max_attempts,
                          int n_f, const FieldDesc* fd_host, swf_precision prec, void* psi_out, cudaStream_t st);
// Breit-Wheeler: march U (fields 2i) and V (fields 2i+1) together and accumulate the appended
// integral M(t) of Eq. 34.  photon_host: per instance k[3], eps[3].
// form 1: the integrand of Eq. 17 for (ss, bs, sb) into macc [n_inst][3] (M_finite = -M(t_in)).
// form 2: the partial-integration integrand of Eqs. 30-33 into macc [n_inst][9]: the mode sum of
//   the ss term, then the time-weighted direct transforms D_U[4] of -iV(U_scat + U_back) at
//   k - q and D_V[4] of -iV(V_scat + V_back) at p - k (wave_k_host: per wave the momentum of its
//   direct transform, 3 doubles; bw_finalize_partial turns these into amplitudes).
swf_status march_bw(swf_ctx* ctx, const GridDesc& g, double t_in, double t_out, int n_steps, int n_inst,
                    const FieldDesc* fd_host, const double* photon_host, swf_precision prec, void* psi_out,
                    double2* macc, cudaStream_t st, int form = 1, const double* wave_k_host = nullptr,
                    int n_ph = 1);
// The same march (form 1, one photon per instance) with step-size control (first step h0, at most
// max_attempts attempts; tolerances from ctx); macc [n_inst][3].
swf_status march_bw_adaptive(swf_ctx* ctx, const GridDesc& g, double t_in, double t_out, double h0, int max_attempts,
                             int n_inst, const FieldDesc* fd_host, const double* photon_host, swf_precision prec,
                             void* psi_out, double2* macc, cudaStream_t st);
// (n_ph photons per instance, form 1 only: photon_host and macc then hold n_inst * n_ph entries,
// photon j of instance i at i n_ph + j; the marched waves are shared by the photons.)

// Breit-Wheeler past terms and totals (swf_bw.cu).
size_t bw_inst_size();
void bw_fill_inst(void* dst, const swf_instance& in, int out, const FieldDesc& fu, const FieldDesc& fv,
                  const int shift[3], int src);
swf_status bw_finalize(swf_ctx* ctx, const GridDesc& g, int n_inst, const void* bw_host, double t_in,
                       const double2* spec, const double2* tat, const double2* macc, const double* norms,
                       swf_result* results, cudaStream_t st);
// sum_j w_j amp_j of n results (4 complex: the three terms and M); weights_host [n] complex.
swf_status bw_packet(swf_ctx* ctx, int n, const swf_result* results, const double* weights_host, double2* out,
                     cudaStream_t st);
swf_status bw_finalize_partial(swf_ctx* ctx, const GridDesc& g, int n_inst, const void* bw_host,
                               const double2* macc, const double* norms, swf_result* results, cudaStream_t st);

// Multi-grid march: groups of fields on different grids sharing one time grid, marched by one
// launch per pass for all groups (persistent blocks on a device work queue) and one CUDA graph
// per step pair.  Each group's result is bitwise that of marching it alone.
struct MultiGroup {
  GridDesc g;
  int F;                  // fields (Breit-Wheeler: 2 per instance, U then V)
  const FieldDesc* fd;    // host, F descriptors
  void* psi_out;          // device, psi(t_in) [F][4][N] in the march precision
  const double* photon;   // Breit-Wheeler: host, per instance k[3], eps[3]; else null
  double2* macc;          // Breit-Wheeler: device, per instance the three integrals of Eq. 17
};
// Groups may be combined when they have the same non-trivial axes (2D with 2D, 3D with 3D).
bool multi_compatible(const GridDesc& a, const GridDesc& b);
// bw = 1: Breit-Wheeler (form 1, one photon per instance) with the integrand of Eq. 17.
swf_status march_multi(swf_ctx* ctx, const std::vector<MultiGroup>& groups, double t_in, double t_out, int n_steps,
                       swf_precision prec, int bw, cudaStream_t st);
// Plain marches of several groups, with the spin reuse of march_fields within each group.
swf_status march_fields_multi(swf_ctx* ctx, const std::vector<MultiGroup>& groups, double t_in, double t_out,
                              int n_steps, swf_precision prec, cudaStream_t st);

// ---- fused cluster march (swf_fused.cu)
bool fused_applicable(const GridDesc& g, int n_f, const FieldDesc* fd, swf_precision prec);
swf_status march_fused(swf_ctx* ctx, const GridDesc& g, double t_in, double t_out, int n_steps, int n_f,
                       const FieldDesc* fd_host, void* psi_out, cudaStream_t st);
// Clusters of the fused kernel resident at once on this device (sets the kernel up on first use);
// 0 if it cannot be resident.
int fused_resident_clusters(swf_ctx* ctx);
// Fields of an n_f-field fused march to give to the pass kernels running concurrently on the SMs
// that the 16-CTA clusters leave free (0: no split).
int fused_split_count(int n_f, int ncl, int n_sm, int variant = kDefaultFusedVariant);
swf_status rhs_eval(swf_ctx* ctx, const GridDesc& g, const FieldDesc& fd, swf_precision prec,
                    double t, const void* psi, void* out, cudaStream_t st);
// The same evaluation with all workspace taken from caller-provided device scratch.
size_t rhs_scratch_bytes(const GridDesc& g, swf_precision prec);
swf_status rhs_eval_scratch(const GridDesc& g, const FieldDesc& fd, swf_precision prec, double t, const void* psi,
                            void* out, void* scratch, cudaStream_t st);

// ---- projections (swf_project.cu)
// psi [F][4][N] (march precision) -> FP64 transform on every grid mode, with the continuum
// normalisation dx^d and the grid-origin phase: spec [F][4][N] double2.
swf_status transform_fields(swf_ctx* ctx, const GridDesc& g, int n_f, swf_precision prec,
                            const void* psi, double2* spec, cudaStream_t st);
// C-spectrum from electron-wave transforms: c_out [F][2][N] double2, prob [F][2][N].
swf_status c_spectrum(swf_ctx* ctx, const GridDesc& g, int n_f, const FieldDesc* fd_host,
                      double t_in, const double2* spec, double2* c_out, double* prob,
                      cudaStream_t st);
// Direct FP64 transform of each field at one wave vector per field: out [F][4] double2.
swf_status transform_at(swf_ctx* ctx, const GridDesc& g, int n_f, swf_precision prec,
                        const void* psi, const double* kappa_host /* [F][3] */, double2* out,
                        cudaStream_t st);
// ||psi_f||^2 (grid inner product) per field: out [F].
swf_status field_norms(swf_ctx* ctx, const GridDesc& g, int n_f, swf_precision prec,
                       const void* psi, double* out, cudaStream_t st);

}  // namespace swf
