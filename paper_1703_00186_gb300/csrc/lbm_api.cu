// C ABI of liblbm.so: contexts, argument checking and kernel launches.
// Declarations and their documentation: include/lbm.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>

#include "lbm_internal.h"

namespace lbm {
cudaError_t launch_step(int prec, bool collide, const void* src, void* dst, const LatticeArgs& a,
                        cudaStream_t s);
cudaError_t launch_init(int prec, void* dst, const double* rho, const double* ux, const double* uy,
                        const double* T, const LatticeArgs& a, cudaStream_t s);
cudaError_t launch_moments(int prec, const void* src, double* rho, double* ux, double* uy, double* T,
                           const LatticeArgs& a, cudaStream_t s);
cudaError_t launch_finite(int prec, const void* src, const LatticeArgs& a, unsigned int* flag,
                          cudaStream_t s);
cudaError_t launch_profiles(int prec, const void* src, double* out, const LatticeArgs& a, cudaStream_t s);
cudaError_t launch_step_observe(const void* src, void* dst, const LatticeArgs& a, double* obs, cudaStream_t s);
bool step_uses_tma(const LatticeArgs& a, const void* src);
cudaError_t launch_step_columns(int prec, bool collide, const void* src, void* dst, const LatticeArgs& a, int x0,
                                int x1, cudaStream_t s);
cudaError_t launch_columns_copy(int prec, bool pack, const void* from, void* to, const LatticeArgs& a, int x0, int n,
                                cudaStream_t s);
cudaError_t launch_adjoint(int prec, const void* f_t, const double* lam_in, double* lam_out,
                           const LatticeArgs& a, cudaStream_t s);
cudaError_t launch_moments_vjp(int prec, const void* f, const double* g_rho, const double* g_ux,
                               const double* g_uy, const double* g_T, double* lam_out,
                               const LatticeArgs& a, cudaStream_t s);
cudaError_t launch_adjoint_f32(const void* f_t, const float* lam_in, float* lam_out, const LatticeArgs& a,
                               cudaStream_t s);
cudaError_t launch_moments_vjp_f32(int prec, const void* f, const double* g_rho, const double* g_ux,
                                   const double* g_uy, const double* g_T, float* lam_out, const LatticeArgs& a,
                                   cudaStream_t s);
cudaError_t launch_init_vjp_f32(const double* rho, const double* ux, const double* uy, const double* T,
                                const float* lam, double* g_rho, double* g_ux, double* g_uy, double* g_T,
                                const LatticeArgs& a, cudaStream_t s);
cudaError_t launch_init_vjp(const double* rho, const double* ux, const double* uy, const double* T,
                            const double* lam, double* g_rho, double* g_ux, double* g_uy,
                            double* g_T, const LatticeArgs& a, cudaStream_t s);

namespace {
std::once_flag g_quad_once;
Quadrature g_quad;
int g_quad_rc = -1;
char g_quad_err[256] = "";

const Quadrature* quadrature(char* err, size_t errlen) {
  std::call_once(g_quad_once, [] { g_quad_rc = solve_quadrature(&g_quad, g_quad_err, sizeof g_quad_err); });
  if (g_quad_rc != 0) {
    std::snprintf(err, errlen, "%s", g_quad_err);
    return nullptr;
  }
  return &g_quad;
}
}  // namespace

size_t element_size(int precision);

// sum_i k_i v_i, exactly, as a 96-bit two's-complement number on the 2^-82
// grid (words w0, w1, w2 as the device's Fix96), for float64 values |v_i| < 4
// and small integer weights k_i.  Bits of a value below 2^-82 are dropped.
static void fix_words(const double* v, const int* k, int n, unsigned out[3]) {
  __int128 acc = 0;
  for (int i = 0; i < n; ++i) {
    if (v[i] == 0.0 || k[i] == 0) continue;
    int e = 0;
    const double m = std::frexp(std::fabs(v[i]), &e);         // |v| = m 2^e, m in [0.5, 1)
    const long long M = (long long)std::ldexp(m, 53);          // exact 53-bit integer
    const int sh = e - 53 + 82;                                // |v| 2^82 = M 2^sh
    __int128 t = sh >= 0 ? ((__int128)M << sh) : (sh > -64 ? (__int128)(M >> -sh) : 0);
    if (v[i] < 0) t = -t;
    acc += t * k[i];
  }
  const unsigned __int128 u = (unsigned __int128)acc;
  out[0] = (unsigned)(u & 0xffffffffu);
  out[1] = (unsigned)((u >> 32) & 0xffffffffu);
  out[2] = (unsigned)((u >> 64) & 0xffffffffu);
}

// Fill the per-launch constants of a lattice.  Returns 0 or an error code
// with a message in err.
int make_lattice_args(const lbm_params& p, LatticeArgs* a, char* err, size_t errlen) {
  if (p.lx < 3 || p.ly < 6) {
    std::snprintf(err, errlen, "lattice %d x %d too small (need lx >= 3, ly >= 6)", p.lx, p.ly);
    return LBM_ERR_INVALID;
  }
  if ((long long)p.lx * (p.ly + 2 * HALO) > (1LL << 40) || p.ly > 4 * 65535) {
    std::snprintf(err, errlen, "lattice too large (ly <= 262140, lx * (ly + 6) <= 2^40)");
    return LBM_ERR_INVALID;
  }
  if (p.precision != LBM_FP64 && p.precision != LBM_FP32_SHIFTED && p.precision != LBM_FP64_DF) {
    std::snprintf(err, errlen, "unknown precision %d", p.precision);
    return LBM_ERR_INVALID;
  }
  if (!(p.tau > 0.5) || !std::isfinite(p.tau) || !std::isfinite(p.g) || !std::isfinite(p.t_top) ||
      !std::isfinite(p.t_bottom) || !std::isfinite(p.rho0) || !(p.t_top > 0) || !(p.t_bottom > 0)) {
    std::snprintf(err, errlen, "invalid physical parameters (need tau > 0.5, finite g, T_wall > 0)");
    return LBM_ERR_INVALID;
  }
  if (p.flags & ~(LBM_FLAG_PERIODIC_Y | LBM_FLAG_REGULARIZED | LBM_FLAG_TMA_LOADS | LBM_FLAG_FP32_F64_TERMS |
                  LBM_FLAG_FP32_F64_COLLIDE)) {
    std::snprintf(err, errlen, "unknown flags 0x%x", p.flags);
    return LBM_ERR_INVALID;
  }
  const int f32_flags = p.flags & (LBM_FLAG_FP32_F64_TERMS | LBM_FLAG_FP32_F64_COLLIDE);
  if (f32_flags && (p.precision != LBM_FP32_SHIFTED || f32_flags == (LBM_FLAG_FP32_F64_TERMS | LBM_FLAG_FP32_F64_COLLIDE))) {
    std::snprintf(err, errlen, "LBM_FLAG_FP32_F64_TERMS / _COLLIDE: one of them, LBM_FP32_SHIFTED only");
    return LBM_ERR_INVALID;
  }
  if ((p.flags & LBM_FLAG_REGULARIZED) && p.precision != LBM_FP64) {
    std::snprintf(err, errlen, "the regularised collide is implemented for LBM_FP64 only");
    return LBM_ERR_INVALID;
  }
  const Quadrature* q = quadrature(err, errlen);
  if (!q) return LBM_ERR_INVALID;
  std::memset(a, 0, sizeof *a);
  a->lx = p.lx;
  a->ly = p.ly;
  a->plane = (long long)(p.ly + 2 * HALO) * p.lx;
  a->idx32 = (long long)NPOP * a->plane < (1LL << 31) ? 1 : 0;
  if (a->idx32) {
    const long long es = (long long)element_size(p.precision);
    for (int l = 0; l < NPOP; ++l) {
      a->plane_off[l] = l * a->plane * es;
      a->pull_off[l] = (l * a->plane - (long long)vy(l) * p.lx - vx(l)) * es;
    }
  }
  a->periodic_y = (p.flags & LBM_FLAG_PERIODIC_Y) ? 1 : 0;
  a->regularized = (p.flags & LBM_FLAG_REGULARIZED) ? 1 : 0;
  a->tma_loads = (p.flags & LBM_FLAG_TMA_LOADS) ? 1 : 0;
  a->fp32_arith = (p.flags & LBM_FLAG_FP32_F64_TERMS)     ? FP32_ARITH_F64_TERMS
                  : (p.flags & LBM_FLAG_FP32_F64_COLLIDE) ? FP32_ARITH_F64_COLLIDE
                                                          : FP32_ARITH_SPLIT;
  a->tau = p.tau;
  a->g = p.g;
  a->omega = 1.0 / p.tau;
  a->omc = 1.0 - a->omega;
  a->r = q->r;
  a->r2 = q->r * q->r;
  a->r2_2 = 0.5 * a->r2;
  a->r2_4 = 0.25 * a->r2;
  a->r4_4 = 0.25 * (a->r2 * a->r2);
  a->r4_8 = 0.125 * (a->r2 * a->r2);
  a->inv_r2 = q->y;
  a->tau_g_xi = p.tau * p.g / q->r;
  a->tshift = p.tau * (1.0 - p.tau) * p.g * p.g / 2.0 - 1.0;
  a->r2_tau_g_xi = a->r2 * a->tau_g_xi;
  a->tshift_v = a->tshift - a->r2_2 * a->tau_g_xi * a->tau_g_xi;
  a->half_inv_r2 = 0.5 * a->inv_r2;
  a->quarter_inv_r2 = 0.25 * a->inv_r2;
  a->inv_r = 1.0 / q->r;
  a->uy_obs_shift = p.tau * p.g - 0.5 * p.g;
  a->rho0 = p.rho0;
  for (int j = 0; j < NSHELL; ++j) {
    a->w_shell[j] = q->w_shell[j];
    a->c2_shell[j] = q->c2_shell[j];
    a->c2h_shell[j] = 0.5 * q->c2_shell[j];
    a->c2q_shell[j] = 0.25 * q->c2_shell[j];
    a->c4e_shell[j] = 0.125 * (q->c2_shell[j] * q->c2_shell[j]);
    a->w6_shell[j] = q->w_shell[j] / 6.0;
  }
  if (a->regularized) {
    if (regularization_gram_inverse(*q, a->ginv) != 0) {
      std::snprintf(err, errlen, "singular Gram matrix");
      return LBM_ERR_INVALID;
    }
    for (double& g : a->ginv) g *= a->omc;  // the collide only needs (1 - omega) G^-1
  }
  wall_ratios(*q, p.t_bottom, 0, a->q_bot);
  wall_ratios(*q, p.t_top, 1, a->q_top);
  for (int l = 0; l < NPOP; ++l) {
    a->w_rho0[l] = q->w[l] * p.rho0;
    a->w_rho0_f[l] = (float)a->w_rho0[l];
  }
  {
    // exact sums of the shift constants on the 2^-82 grid (see fix_words)
    double v_rho[NPOP], v_exi[NPOP];
    for (int l = 0; l < NPOP; ++l) {
      v_rho[l] = a->w_rho0[l];
      v_exi[l] = a->w_rho0[l];
    }
    int one[NPOP], c2[NPOP];
    for (int l = 0; l < NPOP; ++l) {
      one[l] = 1;
      c2[l] = sq(l);
    }
    fix_words(v_rho, one, NPOP, a->fix_shift_rho);
    fix_words(v_exi, c2, NPOP, a->fix_shift_exi);
  }
  for (int j = 0; j < NSHELL; ++j) a->ow_shell[j] = a->omega * q->w_shell[j];
  for (int j = 0; j < NSHELL; ++j) {
    a->w_shell_f[j] = (float)q->w_shell[j];
    a->c2_shell_f[j] = (float)q->c2_shell[j];
  }
  a->omega_f = (float)a->omega;
  a->omc_f = (float)a->omc;
  auto split = [](double v, float out[2]) {
    out[0] = (float)v;
    out[1] = (float)(v - (double)out[0]);
  };
  split(p.rho0, a->df_rho0);
  split(2.0 * q->y * p.rho0, a->df_e0);
  split(a->r2, a->df_r2);
  split(0.5 * a->r2, a->df_half_r2);
  split(q->y, a->df_inv_r2);
  split(a->tshift, a->df_tshift);
  split(a->tau_g_xi, a->df_taug_r);
  split(p.g / q->r, a->df_g_r);
  split(a->omega, a->df_omega);
  split(a->omc, a->df_omc);
  for (int j = 0; j < NSHELL; ++j) {
    // w and c2 exactly as double-words from the double-double solution
    a->df_w_shell[j][0] = (float)q->w_shell[j];
    a->df_w_shell[j][1] = (float)((q->w_shell[j] - (double)a->df_w_shell[j][0]) + q->w_shell_lo[j]);
    split(q->c2_shell[j], a->df_c2_shell[j]);
  }
  return LBM_OK;
}

size_t element_size(int precision) { return precision == LBM_FP32_SHIFTED ? sizeof(float) : sizeof(double); }

// Storage type of a precision mode (LBM_FP64_DF stores float64).
int storage_prec(int precision) { return precision == LBM_FP32_SHIFTED ? LBM_FP32_SHIFTED : LBM_FP64; }

}  // namespace lbm

using namespace lbm;

struct lbm_ctx {
  lbm_params p;
  LatticeArgs args;
  void* buf[2];
  int cur;
  size_t bytes;
  cudaStream_t stream;
  unsigned int* dev;  // [0] status word, [1] finite flag
  cudaStream_t capture = nullptr;                           // private stream for graph capture
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;   // (n, start buffer) -> n steps
  char err[512];
};

namespace {

int fail(lbm_ctx* c, int code, const char* fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(c->err, sizeof c->err, fmt, ap);
    va_end(ap);
  }
  return code;
}

int cuda_check(lbm_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LBM_OK;
  return fail(c, LBM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

extern "C" {

size_t lbm_state_bytes(const lbm_params* p) {
  if (!p || p->lx < 3 || p->ly < 6) return 0;
  if (p->precision != LBM_FP64 && p->precision != LBM_FP32_SHIFTED && p->precision != LBM_FP64_DF) return 0;
  return (size_t)NPOP * (size_t)(p->ly + 2 * HALO) * (size_t)p->lx * element_size(p->precision);
}

int lbm_create(lbm_ctx** out, const lbm_params* p, void* f_a, void* f_b, size_t bytes, void* stream) {
  if (!out) return LBM_ERR_INVALID;
  *out = nullptr;
  if (!p || !f_a || !f_b || f_a == f_b) return LBM_ERR_INVALID;
  lbm_ctx* c = new (std::nothrow) lbm_ctx();
  if (!c) return LBM_ERR_INVALID;
  c->p = *p;
  int rc = make_lattice_args(*p, &c->args, c->err, sizeof c->err);
  if (rc != LBM_OK) {
    delete c;
    return rc;
  }
  if (bytes != lbm_state_bytes(p)) {
    delete c;
    return LBM_ERR_SIZE;
  }
  if (!aligned(f_a, element_size(p->precision)) || !aligned(f_b, element_size(p->precision))) {
    delete c;
    return LBM_ERR_INVALID;
  }
  c->buf[0] = f_a;
  c->buf[1] = f_b;
  c->cur = 0;
  c->bytes = bytes;
  c->stream = static_cast<cudaStream_t>(stream);
  if (cudaMalloc(&c->dev, 2 * sizeof(unsigned int)) != cudaSuccess) {
    cudaGetLastError();
    delete c;
    return LBM_ERR_CUDA;
  }
  c->args.status = c->dev;
  if (cudaMemsetAsync(c->dev, 0, 2 * sizeof(unsigned int), c->stream) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(c->dev);
    delete c;
    return LBM_ERR_CUDA;
  }
  *out = c;
  return LBM_OK;
}

void lbm_destroy(lbm_ctx* c) {
  if (!c) return;
  if (c->dev) {
    cudaStreamSynchronize(c->stream);
    cudaFree(c->dev);
  }
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  if (c->capture) cudaStreamDestroy(c->capture);
  delete c;
}

const char* lbm_last_error(const lbm_ctx* c) { return c ? c->err : "null context"; }

int lbm_set_stream(lbm_ctx* c, void* stream) {
  if (!c) return LBM_ERR_INVALID;
  c->stream = static_cast<cudaStream_t>(stream);
  return LBM_OK;
}

int lbm_init(lbm_ctx* c, const double* rho, const double* ux, const double* uy, const double* T) {
  if (!c) return LBM_ERR_INVALID;
  if (!rho || !ux || !uy || !T) return fail(c, LBM_ERR_INVALID, "lbm_init: NULL field");
  return cuda_check(c, launch_init(storage_prec(c->p.precision), c->buf[c->cur], rho, ux, uy, T, c->args, c->stream),
                    "lbm_init");
}

int lbm_step(lbm_ctx* c, int n) {
  if (!c) return LBM_ERR_INVALID;
  if (n < 0) return fail(c, LBM_ERR_INVALID, "lbm_step: n < 0");
  for (int i = 0; i < n; ++i) {
    cudaError_t e = launch_step(c->p.precision, true, c->buf[c->cur], c->buf[1 - c->cur], c->args, c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "lbm_step");
    c->cur ^= 1;
  }
  return LBM_OK;
}

int lbm_step_graph(lbm_ctx* c, int n) {
  if (!c) return LBM_ERR_INVALID;
  if (n < 0) return fail(c, LBM_ERR_INVALID, "lbm_step_graph: n < 0");
  if (n == 0) return LBM_OK;
  const auto key = std::make_pair(n, c->cur);
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    if (!c->capture && cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking) != cudaSuccess) {
      c->capture = nullptr;
      return cuda_check(c, cudaGetLastError(), "lbm_step_graph: stream");
    }
    int rc = cuda_check(c, cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal), "lbm_step_graph");
    if (rc) return rc;
    cudaError_t le = cudaSuccess;
    int cur = c->cur;
    for (int i = 0; i < n && le == cudaSuccess; ++i) {
      le = launch_step(c->p.precision, true, c->buf[cur], c->buf[1 - cur], c->args, c->capture);
      cur ^= 1;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(c->capture, &g);
    if (le != cudaSuccess || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_check(c, le != cudaSuccess ? le : ee, "lbm_step_graph: capture");
    }
    cudaGraphExec_t exec = nullptr;
    rc = cuda_check(c, cudaGraphInstantiate(&exec, g, 0), "lbm_step_graph: instantiate");
    cudaGraphDestroy(g);
    if (rc) return rc;
    it = c->graphs.emplace(key, exec).first;
  }
  const int rc = cuda_check(c, cudaGraphLaunch(it->second, c->stream), "lbm_step_graph: launch");
  if (rc) return rc;
  c->cur ^= (n & 1);
  return LBM_OK;
}

int lbm_step_from(lbm_ctx* c, const void* src, void* dst) {
  if (!c) return LBM_ERR_INVALID;
  if (!src || !dst || src == dst) return fail(c, LBM_ERR_INVALID, "lbm_step_from: bad buffers");
  return cuda_check(c, launch_step(c->p.precision, true, src, dst, c->args, c->stream), "lbm_step_from");
}

int lbm_step_columns(lbm_ctx* c, const void* src, void* dst, int x0, int x1) {
  if (!c) return LBM_ERR_INVALID;
  if (!src || !dst || src == dst) return fail(c, LBM_ERR_INVALID, "lbm_step_columns: bad buffers");
  if (x0 < 0 || x1 < x0 || x1 > c->p.lx) return fail(c, LBM_ERR_INVALID, "lbm_step_columns: bad column range");
  return cuda_check(c, launch_step_columns(c->p.precision, true, src, dst, c->args, x0, x1, c->stream),
                    "lbm_step_columns");
}

int lbm_pack_columns(lbm_ctx* c, const void* f, int x0, int n, void* buf) {
  if (!c) return LBM_ERR_INVALID;
  if (!f || !buf) return fail(c, LBM_ERR_INVALID, "lbm_pack_columns: NULL buffer");
  if (x0 < 0 || n < 0 || x0 + n > c->p.lx) return fail(c, LBM_ERR_INVALID, "lbm_pack_columns: bad column range");
  return cuda_check(c, launch_columns_copy(storage_prec(c->p.precision), true, f, buf, c->args, x0, n, c->stream),
                    "lbm_pack_columns");
}

int lbm_unpack_columns(lbm_ctx* c, const void* buf, int x0, int n, void* f) {
  if (!c) return LBM_ERR_INVALID;
  if (!f || !buf) return fail(c, LBM_ERR_INVALID, "lbm_unpack_columns: NULL buffer");
  if (x0 < 0 || n < 0 || x0 + n > c->p.lx) return fail(c, LBM_ERR_INVALID, "lbm_unpack_columns: bad column range");
  return cuda_check(c, launch_columns_copy(storage_prec(c->p.precision), false, buf, f, c->args, x0, n, c->stream),
                    "lbm_unpack_columns");
}

void* lbm_current(const lbm_ctx* c) { return c ? c->buf[c->cur] : nullptr; }

int lbm_swap(lbm_ctx* c) {
  if (!c) return LBM_ERR_INVALID;
  c->cur ^= 1;
  return LBM_OK;
}

int lbm_step_path(const lbm_ctx* c) {
  if (!c) return LBM_ERR_INVALID;
  if (c->p.precision != LBM_FP32_SHIFTED) return LBM_PATH_PLAIN;
  return step_uses_tma(c->args, c->buf[c->cur]) && step_uses_tma(c->args, c->buf[1 - c->cur]) ? LBM_PATH_TMA
                                                                                               : LBM_PATH_PLAIN;
}

int lbm_moments(lbm_ctx* c, const void* f, double* rho, double* ux, double* uy, double* T) {
  if (!c) return LBM_ERR_INVALID;
  if (!rho && !ux && !uy && !T) return fail(c, LBM_ERR_INVALID, "lbm_moments: no output");
  if (!f) f = c->buf[c->cur];
  return cuda_check(c, launch_moments(storage_prec(c->p.precision), f, rho, ux, uy, T, c->args, c->stream), "lbm_moments");
}

int lbm_profiles(lbm_ctx* c, const void* f, double* out) {
  if (!c) return LBM_ERR_INVALID;
  if (!out) return fail(c, LBM_ERR_INVALID, "lbm_profiles: NULL output");
  if (!f) f = c->buf[c->cur];
  return cuda_check(c, launch_profiles(storage_prec(c->p.precision), f, out, c->args, c->stream), "lbm_profiles");
}

int lbm_step_observe(lbm_ctx* c, int n, int every, double* out, int* records) {
  if (!c) return LBM_ERR_INVALID;
  if (n < 0 || every < 1 || (n >= every && !out)) return fail(c, LBM_ERR_INVALID, "lbm_step_observe: bad arguments");
  if (c->p.precision != LBM_FP64 || c->args.regularized)
    return fail(c, LBM_ERR_INVALID, "lbm_step_observe: plain LBM_FP64 contexts only");
  int rec = 0;
  for (int i = 1; i <= n; ++i) {
    cudaError_t e;
    if (i % every == 0) {
      e = launch_step_observe(c->buf[c->cur], c->buf[1 - c->cur], c->args,
                              out + (size_t)rec * LBM_NOBS * (size_t)c->p.ly, c->stream);
      ++rec;
    } else {
      e = launch_step(c->p.precision, true, c->buf[c->cur], c->buf[1 - c->cur], c->args, c->stream);
    }
    if (e != cudaSuccess) return cuda_check(c, e, "lbm_step_observe");
    c->cur ^= 1;
  }
  if (records) *records = rec;
  return LBM_OK;
}

int lbm_get_state(lbm_ctx* c, void* dst) {
  if (!c) return LBM_ERR_INVALID;
  if (!dst) return fail(c, LBM_ERR_INVALID, "lbm_get_state: NULL");
  return cuda_check(c, cudaMemcpyAsync(dst, c->buf[c->cur], c->bytes, cudaMemcpyDefault, c->stream),
                    "lbm_get_state");
}

int lbm_set_state(lbm_ctx* c, const void* src) {
  if (!c) return LBM_ERR_INVALID;
  if (!src) return fail(c, LBM_ERR_INVALID, "lbm_set_state: NULL");
  return cuda_check(c, cudaMemcpyAsync(c->buf[c->cur], src, c->bytes, cudaMemcpyDefault, c->stream),
                    "lbm_set_state");
}

int lbm_propagate_bc(lbm_ctx* c, const void* src, void* dst) {
  if (!c) return LBM_ERR_INVALID;
  if (!src || !dst || src == dst) return fail(c, LBM_ERR_INVALID, "lbm_propagate_bc: bad buffers");
  return cuda_check(c, launch_step(storage_prec(c->p.precision), false, src, dst, c->args, c->stream), "lbm_propagate_bc");
}

int lbm_adjoint_step(lbm_ctx* c, const void* f_t, const double* lam_in, double* lam_out) {
  if (!c) return LBM_ERR_INVALID;
  if (!f_t || !lam_in || !lam_out || (const void*)lam_in == (const void*)lam_out)
    return fail(c, LBM_ERR_INVALID, "lbm_adjoint_step: bad buffers");
  if (c->args.regularized)
    return fail(c, LBM_ERR_INVALID, "lbm_adjoint_step: no adjoint of the regularised collide");
  return cuda_check(c, launch_adjoint(c->p.precision, f_t, lam_in, lam_out, c->args, c->stream),
                    "lbm_adjoint_step");
}

int lbm_moments_vjp(lbm_ctx* c, const void* f, const double* g_rho, const double* g_ux, const double* g_uy,
                    const double* g_T, double* lam_out) {
  if (!c) return LBM_ERR_INVALID;
  if (!f || !lam_out) return fail(c, LBM_ERR_INVALID, "lbm_moments_vjp: bad buffers");
  return cuda_check(c, launch_moments_vjp(storage_prec(c->p.precision), f, g_rho, g_ux, g_uy, g_T, lam_out, c->args, c->stream),
                    "lbm_moments_vjp");
}

int lbm_init_vjp(lbm_ctx* c, const double* rho, const double* ux, const double* uy, const double* T,
                 const double* lam, double* g_rho, double* g_ux, double* g_uy, double* g_T) {
  if (!c) return LBM_ERR_INVALID;
  if (!rho || !ux || !uy || !T || !lam) return fail(c, LBM_ERR_INVALID, "lbm_init_vjp: NULL input");
  return cuda_check(c, launch_init_vjp(rho, ux, uy, T, lam, g_rho, g_ux, g_uy, g_T, c->args, c->stream),
                    "lbm_init_vjp");
}

int lbm_adjoint_step_f32(lbm_ctx* c, const void* f_t, const float* lam_in, float* lam_out) {
  if (!c) return LBM_ERR_INVALID;
  if (c->p.precision != LBM_FP32_SHIFTED)
    return fail(c, LBM_ERR_INVALID, "lbm_adjoint_step_f32: LBM_FP32_SHIFTED contexts only");
  if (!f_t || !lam_in || !lam_out || (const void*)lam_in == (const void*)lam_out)
    return fail(c, LBM_ERR_INVALID, "lbm_adjoint_step_f32: bad buffers");
  if (c->args.regularized)
    return fail(c, LBM_ERR_INVALID, "lbm_adjoint_step_f32: no adjoint of the regularised collide");
  return cuda_check(c, launch_adjoint_f32(f_t, lam_in, lam_out, c->args, c->stream), "lbm_adjoint_step_f32");
}

int lbm_moments_vjp_f32(lbm_ctx* c, const void* f, const double* g_rho, const double* g_ux, const double* g_uy,
                        const double* g_T, float* lam_out) {
  if (!c) return LBM_ERR_INVALID;
  if (!f || !lam_out) return fail(c, LBM_ERR_INVALID, "lbm_moments_vjp_f32: bad buffers");
  return cuda_check(c,
                    launch_moments_vjp_f32(storage_prec(c->p.precision), f, g_rho, g_ux, g_uy, g_T, lam_out, c->args,
                                           c->stream),
                    "lbm_moments_vjp_f32");
}

int lbm_init_vjp_f32(lbm_ctx* c, const double* rho, const double* ux, const double* uy, const double* T,
                     const float* lam, double* g_rho, double* g_ux, double* g_uy, double* g_T) {
  if (!c) return LBM_ERR_INVALID;
  if (!rho || !ux || !uy || !T || !lam) return fail(c, LBM_ERR_INVALID, "lbm_init_vjp_f32: NULL input");
  return cuda_check(c, launch_init_vjp_f32(rho, ux, uy, T, lam, g_rho, g_ux, g_uy, g_T, c->args, c->stream),
                    "lbm_init_vjp_f32");
}

int lbm_check_finite(lbm_ctx* c, const void* f, int* ok) {
  if (!c) return LBM_ERR_INVALID;
  if (!ok) return fail(c, LBM_ERR_INVALID, "lbm_check_finite: NULL ok");
  if (!f) f = c->buf[c->cur];
  int rc = cuda_check(c, cudaMemsetAsync(c->dev + 1, 0, sizeof(unsigned int), c->stream), "lbm_check_finite");
  if (rc) return rc;
  rc = cuda_check(c, launch_finite(storage_prec(c->p.precision), f, c->args, c->dev + 1, c->stream), "lbm_check_finite");
  if (rc) return rc;
  unsigned int flag = 0;
  rc = cuda_check(c, cudaMemcpyAsync(&flag, c->dev + 1, sizeof flag, cudaMemcpyDeviceToHost, c->stream),
                  "lbm_check_finite");
  if (rc) return rc;
  rc = cuda_check(c, cudaStreamSynchronize(c->stream), "lbm_check_finite");
  if (rc) return rc;
  *ok = flag ? 0 : 1;
  return LBM_OK;
}

int lbm_status(lbm_ctx* c) {
  if (!c) return LBM_ERR_INVALID;
  int rc = cuda_check(c, cudaStreamSynchronize(c->stream), "lbm_status");
  if (rc) return rc;
  unsigned int w = 0;
  rc = cuda_check(c, cudaMemcpy(&w, c->dev, sizeof w, cudaMemcpyDeviceToHost), "lbm_status");
  if (rc) return rc;
  if (w) return fail(c, LBM_ERR_TIMEOUT, "device status word 0x%x", w);
  return LBM_OK;
}

int lbm_constants(const lbm_ctx* c, double* r, double* w37, double* q_bottom37, double* q_top37) {
  if (!c) return LBM_ERR_INVALID;
  char err[128];
  const Quadrature* q = quadrature(err, sizeof err);
  if (!q) return LBM_ERR_INVALID;
  if (r) *r = q->r;
  for (int l = 0; l < NPOP; ++l) {
    if (w37) w37[l] = q->w[l];
    if (q_bottom37) q_bottom37[l] = c->args.q_bot[l];
    if (q_top37) q_top37[l] = c->args.q_top[l];
  }
  return LBM_OK;
}

int lbm_model_constants(const lbm_params* p, double* r, double* w37, double* q_bottom37, double* q_top37) {
  if (!p) return LBM_ERR_INVALID;
  LatticeArgs a;
  char err[256];
  const int rc = make_lattice_args(*p, &a, err, sizeof err);
  if (rc != LBM_OK) return rc;
  const Quadrature* q = quadrature(err, sizeof err);
  if (!q) return LBM_ERR_INVALID;
  if (r) *r = q->r;
  for (int l = 0; l < NPOP; ++l) {
    if (w37) w37[l] = q->w[l];
    if (q_bottom37) q_bottom37[l] = a.q_bot[l];
    if (q_top37) q_top37[l] = a.q_top[l];
  }
  return LBM_OK;
}

}  // extern "C"
