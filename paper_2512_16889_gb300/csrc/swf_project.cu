// Projections at t_in (Sec. II, Eqs. 8-9) in FP64: grid transforms of the scattered waves,
// the C-spectrum (U_scat(m) | V_back(r, q)) over every grid positron, direct transforms at
// off-grid wave vectors, and grid norms.
#include <cstring>

#include "swf_internal.h"

namespace swf {

namespace {

constexpr int kT = 256;
constexpr int kMaxE = 20;  // FP64 elements a thread holds per FFT pass

template <typename Rin>
__global__ void k_to_double(const cpx<Rin>* __restrict__ in, cpx<double>* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = cvt<double>(in[i]);
}

// Forward FFT along `axis` of every component plane (planes = F*4, each of N points).
__global__ void __launch_bounds__(kT) k_fft_axis(cpx<double>* data, GridDesc g, int axis, RadixPlan pl,
                                                 const cpx<double>* __restrict__ tw, int lines) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<double>* buf = reinterpret_cast<cpx<double>*>(smem_raw);
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const size_t plane = (size_t)blockIdx.y * g.N;
  const int na = g.n[axis];
  if (axis == 0) {
    const int nrows = ny * nz;
    const int row0 = blockIdx.x * lines;
    for (int e = threadIdx.x; e < lines * nx; e += blockDim.x) {
      const int j = e / nx, x = e - j * nx;
      buf[j * nx + x] = (row0 + j < nrows) ? data[plane + (size_t)(row0 + j) * nx + x] : mk<double>(0, 0);
    }
    __syncthreads();
    fft_lines<double, kMaxE>(buf, nx, lines, pl, false, tw);
    for (int e = threadIdx.x; e < lines * nx; e += blockDim.x) {
      const int j = e / nx, x = e - j * nx;
      if (row0 + j < nrows) data[plane + (size_t)(row0 + j) * nx + x] = buf[j * nx + x];
    }
    return;
  }
  const int TX = lines;
  const int ntx = (nx + TX - 1) / TX;
  const int xt = blockIdx.x % ntx;
  const int o = blockIdx.x / ntx;
  const size_t base = axis == 1 ? (size_t)o * nx * ny : (size_t)o * nx;
  const size_t stride = axis == 1 ? (size_t)nx : (size_t)nx * ny;
  for (int e = threadIdx.x; e < TX * na; e += blockDim.x) {
    const int m = e / TX, t = e - m * TX;
    const int x = xt * TX + t;
    buf[t * na + m] = x < nx ? data[plane + base + m * stride + x] : mk<double>(0, 0);
  }
  __syncthreads();
  fft_lines<double, kMaxE>(buf, na, TX, pl, false, tw);
  for (int e = threadIdx.x; e < TX * na; e += blockDim.x) {
    const int m = e / TX, t = e - m * TX;
    const int x = xt * TX + t;
    if (x < nx) data[plane + base + m * stride + x] = buf[t * na + m];
  }
}

// Continuum normalisation dx^d and the phase exp(-i kappa.x0) of a grid starting at x0.
__global__ void k_mode_scale(cpx<double>* data, GridDesc g, size_t total) {
  const double cell = g.dx[0] * g.dx[1] * g.dx[2];
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i % g.N);
    const int ix = j % g.n[0];
    const int iy = (j / g.n[0]) % g.n[1];
    const int iz = j / (g.n[0] * g.n[1]);
    const double ph = -(mode_kappa(ix, g.n[0], g.L[0]) * g.x0[0] + mode_kappa(iy, g.n[1], g.L[1]) * g.x0[1] +
                        mode_kappa(iz, g.n[2], g.L[2]) * g.x0[2]);
    double sn, cs;
    sincos(ph, &sn, &cs);
    data[i] = cell * (data[i] * mk<double>(cs, sn));
  }
}

// C(m, (r, q)) = exp(i q0 t_in) sum_a conj(U~_a(-q)) v_{r,a}(q); the positron at mode j has
// q = -kappa_j (trivial axes: kappa = K of the electron wave).
__global__ void k_c_spectrum(const cpx<double>* __restrict__ spec, const FieldDesc* fd, GridDesc g, int F,
                             double t_in, cpx<double>* c_out, double* prob) {
  const size_t total = (size_t)F * g.N;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int f = (int)(i / g.N);
    const int j = (int)(i - (size_t)f * g.N);
    const int ix = j % g.n[0];
    const int iy = (j / g.n[0]) % g.n[1];
    const int iz = j / (g.n[0] * g.n[1]);
    const FieldDesc& F0 = fd[f];
    double q[3];
    q[0] = -(g.n[0] > 1 ? mode_kappa(ix, g.n[0], g.L[0]) : F0.K[0]);
    q[1] = -(g.n[1] > 1 ? mode_kappa(iy, g.n[1], g.L[1]) : F0.K[1]);
    q[2] = -(g.n[2] > 1 ? mode_kappa(iz, g.n[2], g.L[2]) : F0.K[2]);
    const double q0 = energy3(q);
    double sn, cs;
    sincos(q0 * t_in, &sn, &cs);
    const cpx<double> ph = mk<double>(cs, sn);
    const cpx<double>* u = spec + (size_t)f * 4 * g.N + j;
    cpx<double> uc[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) uc[a] = u[(size_t)a * g.N];
#pragma unroll
    for (int ir = 0; ir < 2; ++ir) {
      double v[8];
      spinor_uv(q, ir == 0 ? 1 : -1, true, v);
      cpx<double> acc = mk<double>(0, 0);
#pragma unroll
      for (int a = 0; a < 4; ++a) acc = acc + cdot(uc[a], mk<double>(v[2 * a], v[2 * a + 1]));
      acc = ph * acc;
      const size_t o = ((size_t)f * 2 + ir) * g.N + j;
      if (c_out) c_out[o] = acc;
      if (prob) prob[o] = acc.x * acc.x + acc.y * acc.y;
    }
  }
}

template <typename Rin>
__device__ __forceinline__ cpx<double> ld_d(const void* p, size_t i) {
  return cvt<double>(reinterpret_cast<const cpx<Rin>*>(p)[i]);
}

// One block per field: dx^d sum_x psi_a(x) exp(-i kappa.x) for a = 0..3 (deterministic order).
template <typename Rin>
__global__ void __launch_bounds__(kT) k_transform_at(const void* psi, GridDesc g, const double* kappa,
                                                     cpx<double>* part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<double>* ph = reinterpret_cast<cpx<double>*>(smem_raw);  // nx + ny + nz phases
  __shared__ cpx<double> red[kT / 32][4];
  const int f = blockIdx.y;
  const int nt = g.n[0] + g.n[1] + g.n[2];
  for (int i = threadIdx.x; i < nt; i += blockDim.x) {
    int axis = 0, j = i;
    while (j >= g.n[axis]) { j -= g.n[axis]; ++axis; }
    const double xc = g.n[axis] > 1 ? g.x0[axis] + j * g.dx[axis] : 0.0;
    const double k = g.n[axis] > 1 ? kappa[3 * f + axis] : 0.0;
    double sn, cs;
    sincos(-k * xc, &sn, &cs);
    ph[i] = mk<double>(cs, sn);
  }
  __syncthreads();
  cpx<double> acc[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) acc[a] = mk<double>(0, 0);
  const size_t fo = (size_t)f * 4 * g.N;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < g.N; j += gridDim.x * blockDim.x) {
    const int ix = j % g.n[0];
    const int iy = (j / g.n[0]) % g.n[1];
    const int iz = j / (g.n[0] * g.n[1]);
    const cpx<double> e = ph[ix] * ph[g.n[0] + iy] * ph[g.n[0] + g.n[1] + iz];
#pragma unroll
    for (int a = 0; a < 4; ++a) acc[a] = acc[a] + ld_d<Rin>(psi, fo + (size_t)a * g.N + j) * e;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      acc[a].x += __shfl_down_sync(0xffffffffu, acc[a].x, off);
      acc[a].y += __shfl_down_sync(0xffffffffu, acc[a].y, off);
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < 4; ++a) red[wid][a] = acc[a];
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    cpx<double> s = mk<double>(0, 0);
    for (int w = 0; w < kT / 32; ++w) s = s + red[w][threadIdx.x];
    part[((size_t)f * gridDim.x + blockIdx.x) * 4 + threadIdx.x] = s;
  }
}

// out[f][q] = scale * sum_b part[f][b][q], the parts added in order of b (deterministic).
template <typename T>
__global__ void k_sum_parts(const T* __restrict__ part, int nb, int width, double scale, T* out) {
  const int f = blockIdx.x;
  for (int q = threadIdx.x; q < width; q += blockDim.x) {
    T s{};
    for (int b = 0; b < nb; ++b) s = s + part[((size_t)f * nb + b) * width + q];
    out[(size_t)f * width + q] = scale * s;
  }
}

// Blocks per field of a grid reduction: about four waves of the GPU, at least 8 elements a thread.
int reduction_blocks(size_t elems, int n_f) {
  static int nsm = 0;
  if (nsm == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess || nsm <= 0)
      nsm = 152;
  }
  const size_t by_size = (elems + 8 * kT - 1) / (8 * kT);
  const size_t by_gpu = (4 * (size_t)nsm + n_f - 1) / n_f;
  size_t nb = by_size < by_gpu ? by_size : by_gpu;
  return nb < 1 ? 1 : (int)nb;
}

template <typename Rin>
__global__ void __launch_bounds__(kT) k_norms(const void* psi, GridDesc g, double* part) {
  __shared__ double red[kT / 32];
  const int f = blockIdx.y;
  const size_t fo = (size_t)f * 4 * g.N;
  double acc = 0.0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)4 * g.N; i += (size_t)gridDim.x * blockDim.x) {
    const cpx<double> v = ld_d<Rin>(psi, fo + i);
    acc += v.x * v.x + v.y * v.y;
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kT / 32; ++w) s += red[w];
    part[(size_t)f * gridDim.x + blockIdx.x] = s;
  }
}

bool smem_ready[64] = {false};

swf_status ensure_smem() {
  const int dv = dev_slot();
  if (smem_ready[dv]) return SWF_OK;
  cudaError_t e = cudaFuncSetAttribute(k_fft_axis, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kT * (kMaxE - 4) * (int)sizeof(cpx<double>));
  if (e != cudaSuccess) return cuda_status(e, "cudaFuncSetAttribute(k_fft_axis)");
  smem_ready[dv] = true;
  return SWF_OK;
}

}  // namespace

swf_status transform_fields(swf_ctx* ctx, const GridDesc& g, int n_f, swf_precision prec, const void* psi,
                            double2* spec, cudaStream_t st) {
  swf_status s = ensure_smem();
  if (s != SWF_OK) return s;
  const size_t total = (size_t)n_f * 4 * g.N;
  cpx<double>* d = reinterpret_cast<cpx<double>*>(spec);
  const int nb = (int)((total + kT - 1) / kT < 65536 ? (total + kT - 1) / kT : 65536);
  {
    ProfScope ps(ctx, "k_to_double", st);
    if (prec == SWF_C64) k_to_double<float><<<nb, kT, 0, st>>>((const cpx<float>*)psi, d, total);
    else k_to_double<double><<<nb, kT, 0, st>>>((const cpx<double>*)psi, d, total);
  }
  const int cap = kT * (kMaxE - 4);
  for (int axis = 0; axis < 3; ++axis) {
    const int na = g.n[axis];
    if (na <= 1) continue;
    RadixPlan pl;
    if (!make_radix_plan(na, &pl)) {
      set_error("grid size must factor into 2, 3 and 5");
      return SWF_EINVAL;
    }
    const void* tw = nullptr;
    if ((s = twiddles(ctx, na, 1, &tw)) != SWF_OK) return s;
    int lines = cap / na;
    if (axis == 0) {
      const int nrows = g.n[1] * g.n[2];
      if (lines > nrows) lines = nrows;
      dim3 grid((nrows + lines - 1) / lines, n_f * 4);
      ProfScope ps(ctx, "k_fft_axis", st);
      k_fft_axis<<<grid, kT, (size_t)lines * na * sizeof(cpx<double>), st>>>(d, g, 0, pl, (const cpx<double>*)tw, lines);
    } else {
      if (lines > 16) lines = 16;
      if (lines > g.n[0]) lines = g.n[0];
      const int ntx = (g.n[0] + lines - 1) / lines;
      const int other = axis == 1 ? g.n[2] : g.n[1];
      dim3 grid(ntx * other, n_f * 4);
      ProfScope ps(ctx, "k_fft_axis", st);
      k_fft_axis<<<grid, kT, (size_t)lines * na * sizeof(cpx<double>), st>>>(d, g, axis, pl, (const cpx<double>*)tw, lines);
    }
  }
  {
    ProfScope ps(ctx, "k_mode_scale", st);
    k_mode_scale<<<nb, kT, 0, st>>>(d, g, total);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "transform kernels");
  return SWF_OK;
}

swf_status c_spectrum(swf_ctx* ctx, const GridDesc& g, int n_f, const FieldDesc* fd_host, double t_in,
                      const double2* spec, double2* c_out, double* prob, cudaStream_t st) {
  void* pfd = nullptr;
  swf_status s = ws_get(ctx, "proj.fd", sizeof(FieldDesc) * n_f, &pfd);
  if (s != SWF_OK) return s;
  cudaError_t e = cudaMemcpyAsync(pfd, fd_host, sizeof(FieldDesc) * n_f, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "upload field descriptors");
  const size_t total = (size_t)n_f * g.N;
  const int nb = (int)((total + kT - 1) / kT < 65536 ? (total + kT - 1) / kT : 65536);
  ProfScope ps(ctx, "k_c_spectrum", st);
  k_c_spectrum<<<nb, kT, 0, st>>>((const cpx<double>*)spec, (const FieldDesc*)pfd, g, n_f, t_in,
                                  (cpx<double>*)c_out, prob);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "c-spectrum kernel");
  return SWF_OK;
}

swf_status transform_at(swf_ctx* ctx, const GridDesc& g, int n_f, swf_precision prec, const void* psi,
                        const double* kappa_host, double2* out, cudaStream_t st) {
  void* pk = nullptr;
  swf_status s = ws_get(ctx, "proj.kappa", sizeof(double) * 3 * n_f, &pk);
  if (s != SWF_OK) return s;
  cudaError_t e = cudaMemcpyAsync(pk, kappa_host, sizeof(double) * 3 * n_f, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_status(e, "upload wave vectors");
  const size_t sm = (size_t)(g.n[0] + g.n[1] + g.n[2]) * sizeof(cpx<double>);
  const int nb = reduction_blocks(g.N, n_f);
  void* part = nullptr;
  if ((s = ws_get(ctx, "proj.part", sizeof(cpx<double>) * 4 * (size_t)nb * n_f, &part)) != SWF_OK) return s;
  {
    ProfScope ps(ctx, "k_transform_at", st);
    if (prec == SWF_C64)
      k_transform_at<float><<<dim3(nb, n_f), kT, sm, st>>>(psi, g, (const double*)pk, (cpx<double>*)part);
    else
      k_transform_at<double><<<dim3(nb, n_f), kT, sm, st>>>(psi, g, (const double*)pk, (cpx<double>*)part);
  }
  {
    ProfScope ps(ctx, "k_sum_parts", st);
    k_sum_parts<cpx<double>><<<n_f, 32, 0, st>>>((const cpx<double>*)part, nb, 4, g.dx[0] * g.dx[1] * g.dx[2],
                                                 (cpx<double>*)out);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "direct transform kernel");
  return SWF_OK;
}

swf_status field_norms(swf_ctx* ctx, const GridDesc& g, int n_f, swf_precision prec, const void* psi,
                       double* out, cudaStream_t st) {
  const int nb = reduction_blocks((size_t)4 * g.N, n_f);
  void* part = nullptr;
  swf_status s = ws_get(ctx, "proj.norm_part", sizeof(double) * (size_t)nb * n_f, &part);
  if (s != SWF_OK) return s;
  {
    ProfScope ps(ctx, "k_norms", st);
    if (prec == SWF_C64) k_norms<float><<<dim3(nb, n_f), kT, 0, st>>>(psi, g, (double*)part);
    else k_norms<double><<<dim3(nb, n_f), kT, 0, st>>>(psi, g, (double*)part);
  }
  {
    ProfScope ps(ctx, "k_sum_parts", st);
    k_sum_parts<double><<<n_f, 32, 0, st>>>((const double*)part, nb, 1, g.dx[0] * g.dx[1] * g.dx[2], (double*)out);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_status(e, "norm kernel");
  return SWF_OK;
}

}  // namespace swf
