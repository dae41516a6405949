// LSQR (MB-L2, Eq. 5 with Eq. 6) and FISTA (MB-L1, Eq. 5 with Eq. 7) on the
// device: FP32 vectors, FP64 norms and scalar recurrences, no host
// synchronisation inside the iteration loop.
//
// Reductions are deterministic: each block reduces a fixed grid-stride slice
// in a fixed tree, writes one FP64 partial, and the last block to finish (an
// atomic ticket) sums the partials in index order and runs the scalar update.
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.cuh"

using namespace oam;

namespace {

constexpr int kThreads = 256;

struct Scalars {
  // LSQR
  double alpha, beta, rhobar, phibar, damp;
  double inv_alpha, inv_beta, cx, cw;
  double anorm2, arnorm;
  int iters_done, stop_at;
  // FISTA / power iteration
  double mu, L, lambda, t, inv_norm, sum_a, sum_b;
  unsigned int ticket;
  unsigned int pad;
  double partial_a[kRedBlocks];
  double partial_b[kRedBlocks];
};

// One damp of a Tikhonov sweep: its plane-rotation recurrence and the
// coefficients of its x and w updates (the bidiagonalisation is shared).
struct DampState {
  double damp, rhobar, phibar, cx, cw, anorm2, arnorm;
};
constexpr int kMaxDamps = OAM_MAX_SWEEP;
struct SweepDamps {
  double d[kMaxDamps];
};
struct SweepX {
  float *x[kMaxDamps];
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sum (or max) of one double per thread; result valid in thread 0.
template <bool kMax>
__device__ double block_reduce(double v) {
  __shared__ double sh[kThreads / 32];
  v = kMax ? warp_max(v) : warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = (l < kThreads / 32) ? sh[l] : (kMax ? -INFINITY : 0.0);
    v = kMax ? warp_max(v) : warp_sum(v);
  }
  return v;
}

// Store this block's partial(s); returns true in every thread of the last block,
// whose thread 0 then holds the combined totals in *ta / *tb.
template <bool kMax>
__device__ bool finish_blocks(Scalars *S, double a, double b, double *ta, double *tb) {
  __shared__ bool last;
  a = block_reduce<kMax>(a);
  b = block_reduce<kMax>(b);
  if (threadIdx.x == 0) {
    S->partial_a[blockIdx.x] = a;
    S->partial_b[blockIdx.x] = b;
    __threadfence();
    last = atomicAdd(&S->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double sa = kMax ? -INFINITY : 0.0, sb = kMax ? -INFINITY : 0.0;
  for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) {
    const double pa = ((volatile double *)S->partial_a)[i], pb = ((volatile double *)S->partial_b)[i];
    sa = kMax ? fmax(sa, pa) : sa + pa;
    sb = kMax ? fmax(sb, pb) : sb + pb;
  }
  sa = block_reduce<kMax>(sa);
  sb = block_reduce<kMax>(sb);
  if (threadIdx.x == 0) {
    *ta = sa;
    *tb = sb;
    S->ticket = 0;
  }
  return true;
}

// ------------------------------------------------------------------ generic
// Reset the scalar block (ticket, partials untouched: each reduction writes
// its partials before reading them) and set the solver's starting scalars.
__global__ void k_init_scalars(Scalars *S, double damp, double t, double L, double lambda) {
  S->alpha = S->beta = S->rhobar = S->phibar = 0.0;
  S->inv_alpha = S->inv_beta = S->cx = S->cw = 0.0;
  S->anorm2 = S->arnorm = 0.0;
  S->iters_done = 0;
  S->stop_at = 0x7fffffff;
  S->mu = S->inv_norm = S->sum_a = S->sum_b = 0.0;
  S->damp = damp;
  S->t = t;
  S->L = L;
  S->lambda = lambda;
  S->ticket = 0;
}

// Element loops: every vector the solvers touch is 16-byte aligned, so
// threads stride over float4 groups; the last n % 4 elements go to the first
// threads of the grid.  A group's squares are summed in FP32 (four positive
// terms) and added to the thread's FP64 accumulator.
#define OAM_GROUPS(g, n4) \
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < (n4); g += (size_t)gridDim.x * blockDim.x)
#define OAM_TAIL(i, n) \
  for (size_t i = ((n) & ~size_t(3)) + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (n); \
       i += (size_t)gridDim.x * blockDim.x)

__device__ __forceinline__ float sq4(float4 v) { return v.x * v.x + v.y * v.y + (v.z * v.z + v.w * v.w); }
__device__ __forceinline__ float4 ld4(const float *p, size_t g) { return reinterpret_cast<const float4 *>(p)[g]; }
__device__ __forceinline__ void st4(float *p, size_t g, float4 v) { reinterpret_cast<float4 *>(p)[g] = v; }
__device__ __forceinline__ float4 fma4(float a, float4 x, float4 y) {
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float4 mul4(float4 x, float a) { return make_float4(x.x * a, x.y * a, x.z * a, x.w * a); }

__global__ void k_fill(float *x, size_t n, float v) {
  OAM_GROUPS(g, n / 4) st4(x, g, make_float4(v, v, v, v));
  OAM_TAIL(i, n) x[i] = v;
}

// dst = src * (*scale); skipped when the iteration is past a stop.
__global__ void k_scale(float *dst, const float *src, size_t n, const double *scale, const Scalars *S, int it) {
  if (S && it > S->stop_at) return;
  const float f = (float)*scale;
  OAM_GROUPS(g, n / 4) st4(dst, g, mul4(ld4(src, g), f));
  OAM_TAIL(i, n) dst[i] = src[i] * f;
}

// ------------------------------------------------------------------ LSQR
// sum of squares of x (FP32 groups, FP64 across groups)
__device__ __forceinline__ double sumsq(const float *x, size_t n) {
  double acc = 0;
  OAM_GROUPS(g, n / 4) acc += (double)sq4(ld4(x, g));
  OAM_TAIL(i, n) acc += (double)(x[i] * x[i]);
  return acc;
}

// FP64 products and sums rounded one operation at a time: the LSQR scalar
// code is inlined at several call sites, and a fused multiply-add formed at
// one site but not another would make a sweep's scalars differ from the
// single solve's in the last bit.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double sumsq_rn(double a, double b) { return __dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)); }

// beta_1 = ||s||
__global__ void k_lsqr_beta0(const float *s, size_t n, Scalars *S) {
  const double acc = sumsq(s, n);
  double ta, tb;
  if (finish_blocks<false>(S, acc, 0.0, &ta, &tb) && threadIdx.x == 0) {
    S->beta = sqrt(ta);
    S->inv_beta = S->beta > 0 ? 1.0 / S->beta : 0.0;
    S->stop_at = S->beta > 0 ? 0x7fffffff : -1;
    S->iters_done = 0;
  }
}

// alpha_1 = ||A^T u_1||, rhobar = alpha, phibar = beta (also for each of the
// nd damps of a sweep in D)
__global__ void k_lsqr_alpha0(const float *th, size_t n, Scalars *S, DampState *D, int nd) {
  const double acc = sumsq(th, n);
  double ta, tb;
  if (finish_blocks<false>(S, acc, 0.0, &ta, &tb) && threadIdx.x == 0) {
    S->alpha = sqrt(ta);
    S->inv_alpha = S->alpha > 0 ? 1.0 / S->alpha : 0.0;
    if (!(S->alpha > 0)) S->stop_at = -1;
    S->rhobar = S->alpha;
    S->phibar = S->beta;
    S->anorm2 = S->alpha * S->alpha;
    S->arnorm = S->alpha * S->beta;
    for (int i = 0; i < nd; ++i) {
      D[i].rhobar = S->alpha;
      D[i].phibar = S->beta;
      D[i].anorm2 = S->alpha * S->alpha;
      D[i].arnorm = S->alpha * S->beta;
    }
  }
}

// v = th / alpha, w = v, x = 0
__global__ void k_lsqr_vw0(const float *th, float *v, float *w, float *x, size_t n, const Scalars *S) {
  const float ia = (float)S->inv_alpha;
  OAM_GROUPS(g, n / 4) {
    const float4 t = mul4(ld4(th, g), ia);
    st4(v, g, t);
    st4(w, g, t);
    st4(x, g, make_float4(0.f, 0.f, 0.f, 0.f));
  }
  OAM_TAIL(i, n) {
    const float t = th[i] * ia;
    v[i] = t;
    w[i] = t;
    x[i] = 0.0f;
  }
}

// beta u = A v - alpha u   (u updated in place, unnormalised; beta from its norm)
__global__ void k_lsqr_u(const float *ts, float *u, size_t n, Scalars *S, int it, DampState *D, int nd) {
  if (it > S->stop_at) return;
  const float al = (float)S->alpha;
  double acc = 0;
  OAM_GROUPS(g, n / 4) {
    const float4 v = fma4(-al, ld4(u, g), ld4(ts, g));
    st4(u, g, v);
    acc += (double)sq4(v);
  }
  OAM_TAIL(i, n) {
    const float v = fmaf(-al, u[i], ts[i]);
    u[i] = v;
    acc += (double)(v * v);
  }
  double ta, tb;
  if (finish_blocks<false>(S, acc, 0.0, &ta, &tb) && threadIdx.x == 0) {
    S->beta = sqrt(ta);
    S->inv_beta = S->beta > 0 ? 1.0 / S->beta : 0.0;
    S->anorm2 = __dadd_rn(S->anorm2, sumsq_rn(S->beta, S->damp));
    for (int i = 0; i < nd; ++i) D[i].anorm2 = __dadd_rn(D[i].anorm2, sumsq_rn(S->beta, D[i].damp));
    if (!(S->beta > 0)) S->stop_at = it;
  }
}

// One step's plane rotations (FP64): the first eliminates the damping term,
// the second the sub-diagonal beta; updates (rhobar, phibar) and returns the
// x and w coefficients phi/rho and theta/rho.
__device__ __forceinline__ void lsqr_rotate(double alpha, double beta, double damp, double &rhobar, double &phibar,
                                            double &cx, double &cw, double &arnorm) {
  double rhobar1 = rhobar;
  if (damp > 0) {
    rhobar1 = sqrt(sumsq_rn(rhobar, damp));
    phibar = mul_rn(rhobar / rhobar1, phibar);
  }
  const double rho = sqrt(sumsq_rn(rhobar1, beta));
  const double c = rhobar1 / rho, sn = beta / rho;
  const double theta = mul_rn(sn, alpha);
  rhobar = -mul_rn(c, alpha);
  const double phi = mul_rn(c, phibar);
  phibar = mul_rn(sn, phibar);
  cx = phi / rho;
  cw = theta / rho;
  arnorm = fabs(mul_rn(mul_rn(phibar, alpha), c));
}

// alpha v = A^T u - beta v, then the plane rotations (FP64), for the solve's
// own damp and for each of the nd damps of a sweep in D.
__global__ void k_lsqr_v(const float *th, float *v, size_t n, Scalars *S, int it, DampState *D, int nd) {
  if (it > S->stop_at) return;
  const float be = (float)S->beta;
  double acc = 0;
  OAM_GROUPS(g, n / 4) {
    const float4 t = fma4(-be, ld4(v, g), ld4(th, g));
    st4(v, g, t);
    acc += (double)sq4(t);
  }
  OAM_TAIL(i, n) {
    const float t = fmaf(-be, v[i], th[i]);
    v[i] = t;
    acc += (double)(t * t);
  }
  double ta, tb;
  if (finish_blocks<false>(S, acc, 0.0, &ta, &tb) && threadIdx.x == 0) {
    const double alpha = sqrt(ta);
    S->alpha = alpha;
    S->inv_alpha = alpha > 0 ? 1.0 / alpha : 0.0;
    S->anorm2 = __dadd_rn(S->anorm2, mul_rn(alpha, alpha));
    if (!(alpha > 0) && S->stop_at > it) S->stop_at = it;
    double rhobar = S->rhobar, phibar = S->phibar, cx, cw, arnorm;
    lsqr_rotate(alpha, S->beta, S->damp, rhobar, phibar, cx, cw, arnorm);
    S->rhobar = rhobar;
    S->phibar = phibar;
    S->cx = cx;
    S->cw = cw;
    S->arnorm = arnorm;
    for (int i = 0; i < nd; ++i) {
      D[i].anorm2 = __dadd_rn(D[i].anorm2, mul_rn(alpha, alpha));
      lsqr_rotate(alpha, S->beta, D[i].damp, D[i].rhobar, D[i].phibar, D[i].cx, D[i].cw, D[i].arnorm);
    }
    S->iters_done = it + 1;
  }
}

// v = vhat / alpha; x += (phi/rho) w; w = v - (theta/rho) w
__global__ void k_lsqr_xw(float *v, float *w, float *x, size_t n, const Scalars *S, int it) {
  if (it > S->stop_at) return;
  const float ia = (float)S->inv_alpha, cx = (float)S->cx, cw = (float)S->cw;
  OAM_GROUPS(g, n / 4) {
    const float4 vv = mul4(ld4(v, g), ia), ww = ld4(w, g);
    st4(x, g, fma4(cx, ww, ld4(x, g)));
    st4(w, g, fma4(-cw, ww, vv));
    st4(v, g, vv);
  }
  OAM_TAIL(i, n) {
    const float vv = v[i] * ia;
    const float ww = w[i];
    x[i] = fmaf(cx, ww, x[i]);
    w[i] = fmaf(-cw, ww, vv);
    v[i] = vv;
  }
}

// Sweep start: every damp's state, then v = th / alpha, w_i = v, x_i = 0.
__global__ void k_sweep_init(DampState *D, SweepDamps damps, int nd) {
  const int i = threadIdx.x;
  if (i < nd) D[i] = DampState{damps.d[i], 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
}

__global__ void k_sweep_vw0(const float *th, float *v, float *W, size_t wstride, SweepX X, int nd, size_t n,
                            const Scalars *S) {
  const float ia = (float)S->inv_alpha;
  OAM_GROUPS(g, n / 4) {
    const float4 t = mul4(ld4(th, g), ia);
    st4(v, g, t);
    for (int i = 0; i < nd; ++i) {
      st4(W + i * wstride, g, t);
      st4(X.x[i], g, make_float4(0.f, 0.f, 0.f, 0.f));
    }
  }
  OAM_TAIL(j, n) {
    const float t = th[j] * ia;
    v[j] = t;
    for (int i = 0; i < nd; ++i) {
      W[i * wstride + j] = t;
      X.x[i][j] = 0.0f;
    }
  }
}

// v = vhat / alpha once; then for each damp i: x_i += (phi_i/rho_i) w_i,
// w_i = v - (theta_i/rho_i) w_i (the arithmetic of k_lsqr_xw).
__global__ void k_sweep_xw(float *v, float *W, size_t wstride, SweepX X, int nd, size_t n, const Scalars *S,
                           const DampState *D, int it) {
  if (it > S->stop_at) return;
  __shared__ float2 coef[kMaxDamps];
  if (threadIdx.x < nd) coef[threadIdx.x] = make_float2((float)D[threadIdx.x].cx, (float)D[threadIdx.x].cw);
  __syncthreads();
  const float ia = (float)S->inv_alpha;
  OAM_GROUPS(g, n / 4) {
    const float4 vv = mul4(ld4(v, g), ia);
    for (int i = 0; i < nd; ++i) {
      float *w = W + i * wstride, *x = X.x[i];
      const float4 ww = ld4(w, g);
      st4(x, g, fma4(coef[i].x, ww, ld4(x, g)));
      st4(w, g, fma4(-coef[i].y, ww, vv));
    }
    st4(v, g, vv);
  }
  OAM_TAIL(j, n) {
    const float vv = v[j] * ia;
    for (int i = 0; i < nd; ++i) {
      const float ww = W[i * wstride + j];
      X.x[i][j] = fmaf(coef[i].x, ww, X.x[i][j]);
      W[i * wstride + j] = fmaf(-coef[i].y, ww, vv);
    }
    v[j] = vv;
  }
}

// ------------------------------------------------------------------ FISTA
// mu = ||A^T A v|| / ||v||, inv_norm = 1 / ||A^T A v||
__global__ void k_power_norms(const float *th, const float *v, size_t n, Scalars *S) {
  const double a = sumsq(th, n), b = sumsq(v, n);
  double ta, tb;
  if (finish_blocks<false>(S, a, b, &ta, &tb) && threadIdx.x == 0) {
    const double nt = sqrt(ta), nv = sqrt(tb);
    S->mu = nv > 0 ? nt / nv : 0.0;
    S->inv_norm = nt > 0 ? 1.0 / nt : 0.0;
    S->L = 2.0 * 1.01 * S->mu;
  }
}

// lambda = lambda_rel * max |A^T s|
__global__ void k_lambda_rel(const float *th, size_t n, Scalars *S, double lambda_rel) {
  float m = 0.0f;
  OAM_GROUPS(g, n / 4) {
    const float4 v = ld4(th, g);
    m = fmaxf(m, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
  }
  OAM_TAIL(i, n) m = fmaxf(m, fabsf(th[i]));
  double ta, tb;
  if (finish_blocks<true>(S, (double)m, 0.0, &ta, &tb) && threadIdx.x == 0) S->lambda = lambda_rel * ta;
}

// r = A Y - s
__global__ void k_sub(float *r, const float *s, size_t n) {
  OAM_GROUPS(g, n / 4) {
    const float4 a = ld4(r, g), b = ld4(s, g);
    st4(r, g, make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w));
  }
  OAM_TAIL(i, n) r[i] -= s[i];
}

__device__ __forceinline__ float prox(float z, float thr, int nonneg) {
  return nonneg ? fmaxf(z - thr, 0.0f) : copysignf(fmaxf(fabsf(z) - thr, 0.0f), z);
}

// x_new = prox(Y - (2/L) g, lambda/L); Y = x_new + ((t-1)/t') (x_new - x); x = x_new; t = t'
__global__ void k_fista_step(const float *g, float *Y, float *x, size_t n, Scalars *S, int nonneg) {
  const double t = S->t;
  const double tn = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
  const float mom = (float)((t - 1.0) / tn);
  const float step = (float)(2.0 / S->L), thr = (float)(S->lambda / S->L);
  OAM_GROUPS(q, n / 4) {
    const float4 z = fma4(-step, ld4(g, q), ld4(Y, q)), xo = ld4(x, q);
    const float4 xn = make_float4(prox(z.x, thr, nonneg), prox(z.y, thr, nonneg), prox(z.z, thr, nonneg),
                                  prox(z.w, thr, nonneg));
    st4(Y, q, make_float4(fmaf(mom, xn.x - xo.x, xn.x), fmaf(mom, xn.y - xo.y, xn.y), fmaf(mom, xn.z - xo.z, xn.z),
                          fmaf(mom, xn.w - xo.w, xn.w)));
    st4(x, q, xn);
  }
  OAM_TAIL(i, n) {
    const float z = fmaf(-step, g[i], Y[i]);
    const float xn = prox(z, thr, nonneg);
    const float xo = x[i];
    Y[i] = fmaf(mom, xn - xo, xn);
    x[i] = xn;
  }
  double ta, tb;
  if (finish_blocks<false>(S, 0.0, 0.0, &ta, &tb) && threadIdx.x == 0) S->t = tn;
}

// objective pieces: sum (A x - s)^2 over signals, sum |x| over the volume
__global__ void k_objective(const float *ax, const float *s, size_t ns, const float *x, size_t nv, Scalars *S) {
  double a = 0, b = 0;
  OAM_GROUPS(g, ns / 4) {
    const float4 p = ld4(ax, g), q = ld4(s, g);
    a += (double)sq4(make_float4(p.x - q.x, p.y - q.y, p.z - q.z, p.w - q.w));
  }
  OAM_TAIL(i, ns) {
    const float r = ax[i] - s[i];
    a += (double)(r * r);
  }
  OAM_GROUPS(g, nv / 4) {
    const float4 v = ld4(x, g);
    b += (double)(fabsf(v.x) + fabsf(v.y) + (fabsf(v.z) + fabsf(v.w)));
  }
  OAM_TAIL(i, nv) b += (double)fabsf(x[i]);
  double ta, tb;
  if (finish_blocks<false>(S, a, b, &ta, &tb) && threadIdx.x == 0) {
    S->sum_a = ta;
    S->sum_b = tb;
  }
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

struct WorkLayout {
  size_t scal, sig, vol;
  size_t total(int solver) const {
    return solver == 0 ? scal + 2 * sig + 3 * vol : scal + sig + 3 * vol;
  }
};

WorkLayout layout(const oam_model *m) {
  WorkLayout L;
  L.scal = align256(sizeof(Scalars));
  L.sig = align256(sig_elems(m) * sizeof(float));
  L.vol = align256(vol_elems(m) * sizeof(float));
  return L;
}

int red_grid(const oam_model *m) { return std::min(kRedBlocks, 4 * std::max(1, m->sm_count)); }
int vec_grid(const oam_model *m) { return 8 * std::max(1, m->sm_count); }

}  // namespace

extern "C" oam_status oam_solver_work_bytes(const oam_model *m, int32_t solver, size_t *bytes) {
  if (!m || !bytes || (solver != 0 && solver != 1)) return OAM_ERR_INVALID_ARG;
  *bytes = layout(m).total(solver);
  return OAM_OK;
}

#define OAM_LAUNCH_CHECK() OAM_LAUNCHED()
#define OAM_TRY(expr)               \
  do {                              \
    oam_status _r = (expr);         \
    if (_r != OAM_OK) return _r;    \
  } while (0)

extern "C" oam_status oam_lsqr(const oam_model *m, const float *d_s, float *d_x, const oam_lsqr_opts *opts,
                               oam_lsqr_info *info, void *d_work, size_t work_bytes, void *stream) {
  if (!m || !d_s || !d_x || !opts || !d_work) return OAM_ERR_INVALID_ARG;
  if (opts->iters < 0 || !(opts->damp >= 0) || !std::isfinite(opts->damp)) return OAM_ERR_INVALID_ARG;
  const WorkLayout L = layout(m);
  if (work_bytes < L.total(0) || (reinterpret_cast<uintptr_t>(d_work) & 255)) return OAM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_s) | reinterpret_cast<uintptr_t>(d_x)) & 15) return OAM_ERR_INVALID_ARG;
  cudaStream_t st = as_stream(stream);
  char *base = static_cast<char *>(d_work);
  Scalars *S = reinterpret_cast<Scalars *>(base);
  float *u = reinterpret_cast<float *>(base + L.scal);
  float *ts = reinterpret_cast<float *>(base + L.scal + L.sig);
  float *v = reinterpret_cast<float *>(base + L.scal + 2 * L.sig);
  float *w = reinterpret_cast<float *>(base + L.scal + 2 * L.sig + L.vol);
  float *th = reinterpret_cast<float *>(base + L.scal + 2 * L.sig + 2 * L.vol);
  const size_t ns = sig_elems(m), nv = vol_elems(m);
  const int RG = red_grid(m), VG = vec_grid(m);

  k_init_scalars<<<1, 1, 0, st>>>(S, opts->damp, 1.0, 0.0, 0.0);
  OAM_LAUNCH_CHECK();
  k_lsqr_beta0<<<RG, kThreads, 0, st>>>(d_s, ns, S);
  OAM_LAUNCH_CHECK();
  k_scale<<<VG, kThreads, 0, st>>>(u, d_s, ns, &S->inv_beta, nullptr, 0);
  OAM_LAUNCH_CHECK();
  OAM_TRY(apply_adjoint(m, u, th, st));
  k_lsqr_alpha0<<<RG, kThreads, 0, st>>>(th, nv, S, nullptr, 0);
  OAM_LAUNCH_CHECK();
  k_lsqr_vw0<<<VG, kThreads, 0, st>>>(th, v, w, d_x, nv, S);
  OAM_LAUNCH_CHECK();
  for (int it = 0; it < opts->iters; ++it) {
    OAM_TRY(apply_forward(m, v, ts, st));
    k_lsqr_u<<<RG, kThreads, 0, st>>>(ts, u, ns, S, it, nullptr, 0);
    OAM_LAUNCH_CHECK();
    k_scale<<<VG, kThreads, 0, st>>>(u, u, ns, &S->inv_beta, S, it);
    OAM_LAUNCH_CHECK();
    OAM_TRY(apply_adjoint(m, u, th, st));
    k_lsqr_v<<<RG, kThreads, 0, st>>>(th, v, nv, S, it, nullptr, 0);
    OAM_LAUNCH_CHECK();
    k_lsqr_xw<<<VG, kThreads, 0, st>>>(v, w, d_x, nv, S, it);
    OAM_LAUNCH_CHECK();
  }
  if (info) {
    Scalars h;
    OAM_CUDA_TRY(cudaMemcpyAsync(&h, S, offsetof(Scalars, partial_a), cudaMemcpyDeviceToHost, st));
    OAM_CUDA_TRY(cudaStreamSynchronize(st));
    info->iters_done = h.iters_done;
    info->stop_reason = (h.stop_at != 0x7fffffff) ? 1 : 0;
    info->rnorm = std::fabs(h.phibar);
    info->arnorm = h.arnorm;
    info->anorm = std::sqrt(h.anorm2);
  }
  return OAM_OK;
}

namespace {

// Sweep workspace: scalars, the damp states, u and A v (signals), v and A^T u
// (volumes), then one w per damp.
struct SweepLayout {
  size_t scal, damps, sig, vol;
  size_t total(int nd) const { return scal + damps + 2 * sig + (2 + (size_t)nd) * vol; }
};

SweepLayout sweep_layout(const oam_model *m) {
  const WorkLayout W = layout(m);
  return SweepLayout{W.scal, align256(sizeof(DampState) * kMaxDamps), W.sig, W.vol};
}

}  // namespace

extern "C" oam_status oam_lsqr_sweep_work_bytes(const oam_model *m, int32_t n_damps, size_t *bytes) {
  if (!m || !bytes || n_damps < 1 || n_damps > kMaxDamps) return OAM_ERR_INVALID_ARG;
  *bytes = sweep_layout(m).total(n_damps);
  return OAM_OK;
}

extern "C" oam_status oam_lsqr_sweep(const oam_model *m, const float *d_s, int32_t n_damps, const double *damps,
                                     float *const *d_x, int32_t iters, oam_lsqr_info *infos, void *d_work,
                                     size_t work_bytes, void *stream) {
  if (!m || !d_s || !damps || !d_x || !d_work || iters < 0) return OAM_ERR_INVALID_ARG;
  if (n_damps < 1 || n_damps > kMaxDamps) return OAM_ERR_INVALID_ARG;
  const SweepLayout L = sweep_layout(m);
  if (work_bytes < L.total(n_damps) || (reinterpret_cast<uintptr_t>(d_work) & 255)) return OAM_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(d_s) & 15) return OAM_ERR_INVALID_ARG;
  SweepDamps dv{};
  SweepX X{};
  for (int i = 0; i < n_damps; ++i) {
    if (!(damps[i] >= 0) || !std::isfinite(damps[i])) return OAM_ERR_INVALID_ARG;
    if (!d_x[i] || (reinterpret_cast<uintptr_t>(d_x[i]) & 15)) return OAM_ERR_INVALID_ARG;
    dv.d[i] = damps[i];
    X.x[i] = d_x[i];
  }
  cudaStream_t st = as_stream(stream);
  char *base = static_cast<char *>(d_work);
  Scalars *S = reinterpret_cast<Scalars *>(base);
  DampState *D = reinterpret_cast<DampState *>(base + L.scal);
  char *vec = base + L.scal + L.damps;
  float *u = reinterpret_cast<float *>(vec);
  float *ts = reinterpret_cast<float *>(vec + L.sig);
  float *v = reinterpret_cast<float *>(vec + 2 * L.sig);
  float *th = reinterpret_cast<float *>(vec + 2 * L.sig + L.vol);
  float *W = reinterpret_cast<float *>(vec + 2 * L.sig + 2 * L.vol);
  const size_t wstride = L.vol / sizeof(float);
  const size_t ns = sig_elems(m), nv = vol_elems(m);
  const int RG = red_grid(m), VG = vec_grid(m);

  k_init_scalars<<<1, 1, 0, st>>>(S, 0.0, 1.0, 0.0, 0.0);
  OAM_LAUNCH_CHECK();
  k_sweep_init<<<1, kMaxDamps, 0, st>>>(D, dv, n_damps);
  OAM_LAUNCH_CHECK();
  k_lsqr_beta0<<<RG, kThreads, 0, st>>>(d_s, ns, S);
  OAM_LAUNCH_CHECK();
  k_scale<<<VG, kThreads, 0, st>>>(u, d_s, ns, &S->inv_beta, nullptr, 0);
  OAM_LAUNCH_CHECK();
  OAM_TRY(apply_adjoint(m, u, th, st));
  k_lsqr_alpha0<<<RG, kThreads, 0, st>>>(th, nv, S, D, n_damps);
  OAM_LAUNCH_CHECK();
  k_sweep_vw0<<<VG, kThreads, 0, st>>>(th, v, W, wstride, X, n_damps, nv, S);
  OAM_LAUNCH_CHECK();
  for (int it = 0; it < iters; ++it) {
    OAM_TRY(apply_forward(m, v, ts, st));
    k_lsqr_u<<<RG, kThreads, 0, st>>>(ts, u, ns, S, it, D, n_damps);
    OAM_LAUNCH_CHECK();
    k_scale<<<VG, kThreads, 0, st>>>(u, u, ns, &S->inv_beta, S, it);
    OAM_LAUNCH_CHECK();
    OAM_TRY(apply_adjoint(m, u, th, st));
    k_lsqr_v<<<RG, kThreads, 0, st>>>(th, v, nv, S, it, D, n_damps);
    OAM_LAUNCH_CHECK();
    k_sweep_xw<<<VG, kThreads, 0, st>>>(v, W, wstride, X, n_damps, nv, S, D, it);
    OAM_LAUNCH_CHECK();
  }
  if (infos) {
    Scalars h;
    std::vector<DampState> hd(n_damps);
    OAM_CUDA_TRY(cudaMemcpyAsync(&h, S, offsetof(Scalars, partial_a), cudaMemcpyDeviceToHost, st));
    OAM_CUDA_TRY(cudaMemcpyAsync(hd.data(), D, sizeof(DampState) * n_damps, cudaMemcpyDeviceToHost, st));
    OAM_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < n_damps; ++i) {
      infos[i].iters_done = h.iters_done;
      infos[i].stop_reason = (h.stop_at != 0x7fffffff) ? 1 : 0;
      infos[i].rnorm = std::fabs(hd[i].phibar);
      infos[i].arnorm = hd[i].arnorm;
      infos[i].anorm = std::sqrt(hd[i].anorm2);
    }
  }
  return OAM_OK;
}

extern "C" oam_status oam_l1_fista(const oam_model *m, const float *d_s, float *d_x, const oam_fista_opts *opts,
                                   oam_fista_info *info, void *d_work, size_t work_bytes, void *stream) {
  if (!m || !d_s || !d_x || !opts || !d_work) return OAM_ERR_INVALID_ARG;
  if (opts->iters < 0 || opts->power_iters < 0 || !std::isfinite(opts->lambda) || !std::isfinite(opts->L) ||
      !std::isfinite(opts->lambda_rel))
    return OAM_ERR_INVALID_ARG;
  if (opts->L <= 0 && opts->power_iters < 1) return OAM_ERR_INVALID_ARG;
  if (opts->lambda < 0 && opts->lambda_rel < 0) return OAM_ERR_INVALID_ARG;
  const WorkLayout L = layout(m);
  if (work_bytes < L.total(1) || (reinterpret_cast<uintptr_t>(d_work) & 255)) return OAM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_s) | reinterpret_cast<uintptr_t>(d_x) |
       reinterpret_cast<uintptr_t>(opts->d_power_v0)) & 15)
    return OAM_ERR_INVALID_ARG;
  cudaStream_t st = as_stream(stream);
  char *base = static_cast<char *>(d_work);
  Scalars *S = reinterpret_cast<Scalars *>(base);
  float *Y = reinterpret_cast<float *>(base + L.scal);
  float *th = reinterpret_cast<float *>(base + L.scal + L.vol);
  float *v = reinterpret_cast<float *>(base + L.scal + 2 * L.vol);
  float *ts = reinterpret_cast<float *>(base + L.scal + 3 * L.vol);
  const size_t ns = sig_elems(m), nv = vol_elems(m);
  const int RG = red_grid(m), VG = vec_grid(m);

  k_init_scalars<<<1, 1, 0, st>>>(S, 0.0, 1.0, opts->L, opts->lambda);
  OAM_LAUNCH_CHECK();
  if (opts->L <= 0) {
    if (opts->d_power_v0)
      OAM_CUDA_TRY(cudaMemcpyAsync(v, opts->d_power_v0, nv * sizeof(float), cudaMemcpyDeviceToDevice, st));
    else
      k_fill<<<VG, kThreads, 0, st>>>(v, nv, 1.0f);
    OAM_LAUNCH_CHECK();
    for (int it = 0; it < opts->power_iters; ++it) {
      OAM_TRY(apply_forward(m, v, ts, st));
      OAM_TRY(apply_adjoint(m, ts, th, st));
      k_power_norms<<<RG, kThreads, 0, st>>>(th, v, nv, S);
      OAM_LAUNCH_CHECK();
      k_scale<<<VG, kThreads, 0, st>>>(v, th, nv, &S->inv_norm, nullptr, 0);
      OAM_LAUNCH_CHECK();
    }
  }
  if (opts->lambda < 0) {
    OAM_TRY(apply_adjoint(m, d_s, th, st));
    k_lambda_rel<<<RG, kThreads, 0, st>>>(th, nv, S, opts->lambda_rel);
    OAM_LAUNCH_CHECK();
  }
  k_fill<<<VG, kThreads, 0, st>>>(Y, nv, 0.0f);
  OAM_LAUNCH_CHECK();
  k_fill<<<VG, kThreads, 0, st>>>(d_x, nv, 0.0f);
  OAM_LAUNCH_CHECK();
  for (int it = 0; it < opts->iters; ++it) {
    OAM_TRY(apply_forward(m, Y, ts, st));
    k_sub<<<VG, kThreads, 0, st>>>(ts, d_s, ns);
    OAM_LAUNCH_CHECK();
    OAM_TRY(apply_adjoint(m, ts, th, st));
    k_fista_step<<<RG, kThreads, 0, st>>>(th, Y, d_x, nv, S, opts->nonneg);
    OAM_LAUNCH_CHECK();
  }
  if (opts->compute_objective) {
    OAM_TRY(apply_forward(m, d_x, ts, st));
    k_objective<<<RG, kThreads, 0, st>>>(ts, d_s, ns, d_x, nv, S);
    OAM_LAUNCH_CHECK();
  }
  if (info) {
    Scalars h;
    OAM_CUDA_TRY(cudaMemcpyAsync(&h, S, offsetof(Scalars, partial_a), cudaMemcpyDeviceToHost, st));
    OAM_CUDA_TRY(cudaStreamSynchronize(st));
    info->iters_done = opts->iters;
    info->L = h.L;
    info->lambda = h.lambda;
    info->mu = h.mu;
    info->objective = opts->compute_objective ? h.sum_a + h.lambda * h.sum_b : NAN;
  }
  return OAM_OK;
}

// ---------------------------------------------------------------- no-allocation LSQR
// Some callers cannot call cudaMalloc at solve time: hosts that reserve all
// device memory up front for their own allocator (so a library allocation
// would fail or fragment it), and latency-critical loops where an allocation's
// implicit device synchronisation is not acceptable.  oam_lsqr_noalloc runs
// the same LSQR as oam_lsqr on a fixed workspace that lives in this library's
// static device memory instead of a caller-provided buffer.
namespace {

constexpr size_t kStaticWorkBytes = size_t(32) << 20;  // 32 MiB per GPU that loads the library
__device__ __align__(256) unsigned char g_static_work[kStaticWorkBytes];

constexpr int kMaxDevices = 64;
void *g_static_ptr[kMaxDevices] = {};
std::mutex g_static_mu;

// Device address of g_static_work in the current device's context.  Outside
// stream capture it is looked up on every call (cudaGetSymbolAddress, no
// allocation), so a context that was torn down and created again never gets
// a stale address; during capture the address from the last uncaptured call
// on this device is used, so the first call on a device must come before any
// capture (OAM_ERR_INVALID_ARG otherwise).
oam_status static_work_ptr(cudaStream_t st, void **out) {
  int dev = 0;
  OAM_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return OAM_ERR_UNSUPPORTED;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  OAM_CUDA_TRY(cudaStreamIsCapturing(st, &cap));
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_work) != cudaSuccess || !p) {
      cudaGetLastError();
      return OAM_ERR_CUDA;
    }
    g_static_ptr[dev] = p;
  } else if (!g_static_ptr[dev]) {
    return OAM_ERR_INVALID_ARG;
  }
  *out = g_static_ptr[dev];
  return OAM_OK;
}

}  // namespace

extern "C" oam_status oam_lsqr_noalloc(const oam_model *m, const float *d_s, float *d_x, const oam_lsqr_opts *opts,
                                       oam_lsqr_info *info, void *stream) {
  if (!m || !d_s || !d_x || !opts) return OAM_ERR_INVALID_ARG;
  const size_t need = layout(m).total(0);
  if (need > kStaticWorkBytes) return OAM_ERR_INVALID_ARG;
  void *work = nullptr;
  oam_status rc = static_work_ptr(as_stream(stream), &work);
  if (rc) return rc;
  return oam_lsqr(m, d_s, d_x, opts, info, work, kStaticWorkBytes, stream);
}
