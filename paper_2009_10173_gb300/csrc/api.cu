// C-ABI entry points of liboam.so: argument checks, host-side planning of the
// sensor rings and slab orbits, model lifetime, and dispatch to the kernels.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <numeric>

#include "internal.cuh"

using namespace oam;

namespace {

bool finite_pos(double v) { return std::isfinite(v) && v > 0; }

oam_status check_params(const oam_sensor *s, const oam_grid *g, const oam_eir *e) {
  if (!s || !g || !e) return OAM_ERR_INVALID_ARG;
  if (!finite_pos(s->focal_m) || !finite_pos(s->aperture_m) || !(s->aperture_m < 2 * s->focal_m) ||
      !std::isfinite(s->hole_m) || s->hole_m < 0 || !(s->hole_m < s->aperture_m) || !finite_pos(s->c_mps))
    return OAM_ERR_INVALID_ARG;
  if (s->n_patches <= 0 || s->n_patches % 8 != 0 || s->n_patches > (1 << 20)) return OAM_ERR_INVALID_ARG;
  if (g->px < 1 || g->py < 1 || g->nz < 1 || g->nt < 4 || g->nt % 4 != 0) return OAM_ERR_INVALID_ARG;
  if (g->win < 1 || g->win % 2 == 0 || g->win > 255) return OAM_ERR_INVALID_ARG;
  if (g->px > 65535 || g->py > 65535 || g->nz > 4096 || g->nt > (1 << 16)) return OAM_ERR_INVALID_ARG;
  if (!finite_pos(g->dx_m) || !finite_pos(g->dy_m) || !finite_pos(g->dz_m) || !finite_pos(g->fs_hz) ||
      !std::isfinite(g->z0_rel_m) || std::isinf(g->t0_s))
    return OAM_ERR_INVALID_ARG;
  if (!finite_pos(e->fc_hz) || !finite_pos(e->frac_bw) || !finite_pos(e->trunc_sigma))
    return OAM_ERR_INVALID_ARG;
  return OAM_OK;
}

// Rings uniform in polar angle between the hole edge and the aperture edge;
// ring r holds 8*u_r equal patches, sum u_r = M/8, u_r >= 1 and the remaining
// units follow ring area by largest remainder (equal remainders: inner ring first).
std::vector<Ring> plan_rings(const oam_sensor *s) {
  const double F = s->focal_m;
  const double th_in = std::asin(s->hole_m / (2.0 * F));
  const double th_out = std::asin(s->aperture_m / (2.0 * F));
  const double cap = 2.0 * M_PI * F * F * (std::cos(th_in) - std::cos(th_out));
  const int units = s->n_patches / 8;
  long rings = std::lround((th_out - th_in) * F * std::sqrt(double(s->n_patches) / cap));
  rings = std::max(1L, std::min<long>(rings, units));
  std::vector<Ring> out(rings);
  std::vector<double> rem(rings);
  std::vector<int> u(rings);
  const int spare = units - int(rings);
  int handed = 0;
  for (long r = 0; r < rings; ++r) {
    double a0 = th_in + (th_out - th_in) * r / rings;
    double a1 = th_in + (th_out - th_in) * (r + 1) / rings;
    double c0 = std::cos(a0), c1 = std::cos(a1);
    out[r].cos_mid = 0.5 * (c0 + c1);
    out[r].area = 2.0 * M_PI * F * F * (c0 - c1);
    double share = spare * out[r].area / cap;
    double whole = std::floor(share);
    u[r] = 1 + int(whole);
    rem[r] = share - whole;
    handed += int(whole);
  }
  std::vector<int> order(rings);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return rem[x] > rem[y]; });
  for (int i = 0; i < spare - handed; ++i) u[order[i]] += 1;
  int first = 0;
  for (long r = 0; r < rings; ++r) {
    out[r].count = 8 * u[r];
    out[r].first = first;
    first += out[r].count;
  }
  return out;
}

// Orbits of lateral offsets under the slab's mirror symmetries: (b, a) ~
// (+-b, +-a), and additionally (a, b) when dx == dy (the patch set is
// invariant under x<->y and both mirror images; Results, axial symmetry).
void plan_orbits(oam_model *m) {
  const int R = m->R, W = m->W;
  const bool swap = m->grid.dx_m == m->grid.dy_m;
  std::vector<int> id((R + 1) * (R + 1), -1);
  m->h_orb_b.clear();
  m->h_orb_a.clear();
  for (int p = 0; p <= R; ++p)
    for (int q = 0; q <= R; ++q) {
      int lo = p, hi = q;  // (|b|, |a|)
      if (swap && lo > hi) std::swap(lo, hi);
      int key = lo * (R + 1) + hi;
      if (id[key] < 0) {
        id[key] = int(m->h_orb_b.size());
        m->h_orb_b.push_back(lo);
        m->h_orb_a.push_back(hi);
      }
      id[p * (R + 1) + q] = id[key];
    }
  m->n_orb = int(m->h_orb_b.size());
  m->h_tap_orbit.resize(W * W);
  for (int b = -R; b <= R; ++b)
    for (int a = -R; a <= R; ++a) m->h_tap_orbit[(b + R) * W + (a + R)] = id[std::abs(b) * (R + 1) + std::abs(a)];
}

// Range of d - F over the patch set for every (orbit, depth), on the host.
// Within a ring (polar angle fixed) r.n = r_z cos(theta) + sin(theta) rho
// cos(phi - psi), psi the voxel's azimuth, so the ring's largest and smallest
// distances belong to the patches whose azimuths are nearest psi and psi + pi;
// d - F = (2F r.n + |r|^2) / (d + F) grows with r.n.
void host_ranges(const oam_model *m, const std::vector<Ring> &rings, std::vector<double2> *out) {
  const double F = m->sensor.focal_m;
  const int nz = m->grid.nz;
  out->assign((size_t)m->n_orb * nz, make_double2(INFINITY, -INFINITY));
  // patch normals as the device expands them: phi_m = (2m + 1) pi / count
  std::vector<double> nx, ny, nzv;
  for (const Ring &g : rings) {
    const double sn = std::sqrt(1.0 - g.cos_mid * g.cos_mid);
    for (int j = 0; j < g.count; ++j) {
      const double phi = M_PI * (2.0 * j + 1.0) / g.count;
      nx.push_back(sn * std::cos(phi));
      ny.push_back(sn * std::sin(phi));
      nzv.push_back(g.cos_mid);
    }
  }
  std::vector<int> cand;
  for (int o = 0; o < m->n_orb; ++o) {
    const double rx = m->h_orb_a[o] * m->grid.dx_m, ry = m->h_orb_b[o] * m->grid.dy_m;
    const double psi = std::atan2(ry, rx);
    cand.clear();  // per ring: the patches nearest in azimuth to psi and to psi + pi
    for (const Ring &g : rings)
      for (int side = 0; side < 2; ++side) {
        const long m0 = std::lround((psi + (side ? M_PI : 0.0)) * g.count / (2.0 * M_PI) - 0.5);
        for (long dm = -1; dm <= 1; ++dm) cand.push_back(g.first + (int)(((m0 + dm) % g.count + g.count) % g.count));
      }
    for (int k = 0; k < nz; ++k) {
      const double rz = m->grid.z0_rel_m + k * m->grid.dz_m;
      const double r2 = rx * rx + ry * ry + rz * rz;
      double2 &rg = (*out)[(size_t)o * nz + k];
      for (int j : cand) {
        const double rn = rx * nx[j] + ry * ny[j] + rz * nzv[j];
        const double num = 2.0 * F * rn + r2;
        const double dd = num / (std::sqrt(F * F + num) + F);
        rg.x = std::min(rg.x, dd);
        rg.y = std::max(rg.y, dd);
      }
    }
  }
}

void free_model(oam_model *m, cudaStream_t st) {
  if (!m) return;
  tc_free(m, st);
  fft_free(m, st);
  fir_free(m, st);
  for (cudaEvent_t e : m->prof.pool) cudaEventDestroy(e);
  void *ptrs[] = {m->d_status, m->d_tap_orbit, m->d_patch, m->d_band_lo, m->d_band, m->d_fwd_krange, m->d_fwd_off,
                  m->d_fwd, m->d_adj_nrange, m->d_adj_off, m->d_adj};
  for (void *p : ptrs)
    if (p) cudaFreeAsync(p, st);
  delete m;
}

}  // namespace

namespace oam {
// Defined here because it needs the ring planner: expand rings into patches.
oam_status upload_patches(oam_model *m, cudaStream_t st);
}

__global__ void k_expand_patches(const oam::Ring *rings, int n_rings, Patch *out) {
  int r = blockIdx.x;
  if (r >= n_rings) return;
  const oam::Ring g = rings[r];
  double sin_mid = sqrt(1.0 - g.cos_mid * g.cos_mid);
  double area_mm2 = g.area / g.count * 1e6;
  for (int m = threadIdx.x; m < g.count; m += blockDim.x) {
    double sp, cp;
    sincospi((2.0 * m + 1.0) / g.count, &sp, &cp);  // phi = (m + 1/2) 2 pi / count
    out[g.first + m] = oam::Patch{sin_mid * cp, sin_mid * sp, g.cos_mid, area_mm2};
  }
}

oam_status oam::upload_patches(oam_model *m, cudaStream_t st) {
  std::vector<Ring> rings = plan_rings(&m->sensor);
  m->M = m->sensor.n_patches;
  oam_status rc = dev_alloc(m, &m->d_patch, m->M);
  if (rc) return rc;
  Ring *d_rings = nullptr;
  OAM_CUDA_TRY(cudaMallocAsync((void **)&d_rings, sizeof(Ring) * rings.size(), st));
  OAM_CUDA_TRY(cudaMemcpyAsync(d_rings, rings.data(), sizeof(Ring) * rings.size(), cudaMemcpyHostToDevice, st));
  k_expand_patches<<<int(rings.size()), 256, 0, st>>>(d_rings, int(rings.size()), m->d_patch);
  OAM_LAUNCHED();
  OAM_CUDA_TRY(cudaFreeAsync(d_rings, st));
  return OAM_OK;
}

std::atomic<long long> oam::g_launches{0};

void oam::model_release(oam_model *m, cudaStream_t st) { free_model(m, st); }

oam::ProfScope::ProfScope(const oam_model *m_, cudaStream_t s, bool f) : m(m_), st(s), fwd(f) {
  oam_model::Prof &p = m->prof;
  if (!p.on) return;
  while (p.pool.size() < p.used + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    p.pool.push_back(e);
  }
  first = p.used;
  p.used += 2;
  active = cudaEventRecord(p.pool[first], st) == cudaSuccess;
}

oam::ProfScope::~ProfScope() {
  if (!active) return;
  oam_model::Prof &p = m->prof;
  if (cudaEventRecord(p.pool[first + 1], st) != cudaSuccess) return;
  (fwd ? p.fwd : p.adj).emplace_back(first, first + 1);
}

// ---------------------------------------------------------------- C ABI
extern "C" {

int64_t oam_launch_count(void) { return oam::g_launches.load(); }

oam_status oam_profile_enable(oam_model *m, int32_t enable) {
  if (!m) return OAM_ERR_INVALID_ARG;
  if (cudaDeviceSynchronize() != cudaSuccess) return OAM_ERR_CUDA;
  m->prof.on = enable != 0;
  m->prof.used = 0;
  m->prof.fwd.clear();
  m->prof.adj.clear();
  return OAM_OK;
}

oam_status oam_profile_read(oam_model *m, oam_profile *out) {
  if (!m || !out) return OAM_ERR_INVALID_ARG;
  oam_model::Prof &p = m->prof;
  out->forward_calls = (int64_t)p.fwd.size();
  out->adjoint_calls = (int64_t)p.adj.size();
  out->forward_ms = out->adjoint_ms = 0;
  for (int pass = 0; pass < 2; ++pass)
    for (auto &pr : (pass ? p.adj : p.fwd)) {
      if (cudaEventSynchronize(p.pool[pr.second]) != cudaSuccess) return OAM_ERR_CUDA;
      float ms = 0;
      if (cudaEventElapsedTime(&ms, p.pool[pr.first], p.pool[pr.second]) != cudaSuccess) return OAM_ERR_CUDA;
      (pass ? out->adjoint_ms : out->forward_ms) += ms;
    }
  return OAM_OK;
}

int32_t oam_version(void) { return 100; }

const char *oam_status_string(oam_status s) {
  switch (s) {
    case OAM_OK: return "ok";
    case OAM_ERR_INVALID_ARG: return "invalid argument";
    case OAM_ERR_WINDOW: return "arrivals fall outside the sample window";
    case OAM_ERR_OOM: return "out of memory";
    case OAM_ERR_CUDA: return "CUDA runtime error";
    case OAM_ERR_DEVICE: return "device-side error";
    case OAM_ERR_TIMEOUT: return "device-side wait timed out";
    case OAM_ERR_BUSY: return "busy";
    case OAM_ERR_UNSUPPORTED: return "unsupported option or device";
  }
  return "unknown status";
}

oam_status oam_build_model(const oam_sensor *sensor, const oam_grid *grid, const oam_eir *eir,
                           oam_precision precision, void *stream, oam_model **out) {
  return oam_build_model_ex(sensor, grid, eir, precision, nullptr, stream, out);
}

oam_status oam_build_model_ex(const oam_sensor *sensor, const oam_grid *grid, const oam_eir *eir,
                              oam_precision precision, const oam_model_opts *opts, void *stream, oam_model **out) {
  if (!out) return OAM_ERR_INVALID_ARG;
  *out = nullptr;
  oam_status rc = check_params(sensor, grid, eir);
  if (rc) return rc;
  const int disc = opts ? opts->discretisation : OAM_DISC_POINT;
  if (disc != OAM_DISC_POINT && disc != OAM_DISC_TRILINEAR) return OAM_ERR_INVALID_ARG;
  if (precision != OAM_PREC_FP32 && precision != OAM_PREC_BF16X3 && precision != OAM_PREC_FFT)
    return OAM_ERR_INVALID_ARG;
  int dev = 0, major = 0, minor = 0, sms = 0;
  OAM_CUDA_TRY(cudaGetDevice(&dev));
  OAM_CUDA_TRY(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
  OAM_CUDA_TRY(cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev));
  OAM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (major != 10 || minor != 3) return OAM_ERR_UNSUPPORTED;

  oam_model *m = new (std::nothrow) oam_model();
  if (!m) return OAM_ERR_OOM;
  m->sensor = *sensor;
  m->grid = *grid;
  m->eir = *eir;
  m->precision = precision;
  m->disc = disc;
  m->sm_count = sms;
  m->W = grid->win;
  m->R = (grid->win - 1) / 2;
  const double sig_f = eir->fc_hz * eir->frac_bw / (2.0 * std::sqrt(2.0 * std::log(2.0)));
  m->sigma_s = grid->fs_hz / (2.0 * M_PI * sig_f);
  m->omega = 2.0 * M_PI * eir->fc_hz / grid->fs_hz;
  m->cut = eir->trunc_sigma * m->sigma_s;
  plan_orbits(m);
  cudaStream_t st = as_stream(stream);
  m->alloc_stream = st;
  rc = dev_alloc(m, &m->d_status, 1);
  if (!rc && cudaMemsetAsync(m->d_status, 0, sizeof(int), st) != cudaSuccess) rc = OAM_ERR_CUDA;
  if (!rc) rc = upload_patches(m, st);
  if (!rc) rc = build_slab(m, st);
  if (!rc && precision == OAM_PREC_BF16X3) rc = tc_build(m, st);
  if (!rc && precision == OAM_PREC_FFT) rc = fft_build(m, st);
  if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = OAM_ERR_CUDA;
  if (rc) {
    cudaStreamSynchronize(st);
    cudaGetLastError();
    free_model(m, st);
    cudaStreamSynchronize(st);
    return rc;
  }
  *out = m;
  return OAM_OK;
}

oam_status oam_model_bytes(const oam_sensor *sensor, const oam_grid *grid, const oam_eir *eir,
                           oam_precision precision, size_t *bytes) {
  return oam_model_bytes_ex(sensor, grid, eir, precision, nullptr, bytes);
}

oam_status oam_model_bytes_ex(const oam_sensor *sensor, const oam_grid *grid, const oam_eir *eir,
                              oam_precision precision, const oam_model_opts *opts, size_t *bytes) {
  if (!bytes) return OAM_ERR_INVALID_ARG;
  oam_status rc = check_params(sensor, grid, eir);
  if (rc) return rc;
  if (precision != OAM_PREC_FP32 && precision != OAM_PREC_BF16X3 && precision != OAM_PREC_FFT)
    return OAM_ERR_INVALID_ARG;
  const int disc = opts ? opts->discretisation : OAM_DISC_POINT;
  if (disc != OAM_DISC_POINT && disc != OAM_DISC_TRILINEAR) return OAM_ERR_INVALID_ARG;
  oam_model m;  // host-side plan only: no device memory, no device call
  m.disc = disc;
  m.sensor = *sensor;
  m.grid = *grid;
  m.eir = *eir;
  m.precision = precision;
  m.W = grid->win;
  m.R = (grid->win - 1) / 2;
  const double sig_f = eir->fc_hz * eir->frac_bw / (2.0 * std::sqrt(2.0 * std::log(2.0)));
  m.sigma_s = grid->fs_hz / (2.0 * M_PI * sig_f);
  m.omega = 2.0 * M_PI * eir->fc_hz / grid->fs_hz;
  m.cut = eir->trunc_sigma * m.sigma_s;
  m.M = sensor->n_patches;
  plan_orbits(&m);
  std::vector<double2> ranges;
  host_ranges(&m, plan_rings(sensor), &ranges);
  // two samples of margin per band edge: host and device distances may round
  // a band edge, or the automatic time origin, one sample apart
  if ((rc = plan_bands(&m, ranges, 2))) return rc;
  size_t total = alloc_bytes<int>(1) + alloc_bytes<Patch>(m.M) + slab_plan_bytes(&m), extra = 0;
  if (precision == OAM_PREC_BF16X3) rc = tc_plan_bytes(&m, &extra);
  if (precision == OAM_PREC_FFT) rc = fft_plan_bytes(&m, &extra);
  if (rc) return rc;
  *bytes = total + extra;
  return OAM_OK;
}

oam_status oam_model_free(oam_model *model) {
  if (!model) return OAM_OK;
  cudaDeviceSynchronize();
  free_model(model, nullptr);
  cudaStreamSynchronize(nullptr);
  return OAM_OK;
}

oam_status oam_model_get_info(const oam_model *m, oam_model_info *info) {
  if (!m || !info) return OAM_ERR_INVALID_ARG;
  info->t0_s = m->t0;
  info->n_lo = m->n_lo;
  info->n_hi = m->n_hi;
  info->n_orbits = m->n_orb;
  info->precision = m->precision;
  info->nnz = m->nnz;
  info->flops_per_op = m->flops;
  info->device_bytes = m->bytes;
  info->exec_flops_forward = m->precision == OAM_PREC_FFT ? fft_flops(m) : tc_exec_flops(m, 0);
  info->exec_flops_adjoint = m->precision == OAM_PREC_FFT ? fft_flops(m) : tc_exec_flops(m, 1);
  info->op_bytes = fft_bytes(m);
  info->filter_half_len = m->fir ? fir_half_len(m) : -1;
  info->filter_size = m->fir ? fir_size(m) : 0;
  return OAM_OK;
}

oam_status oam_model_slab_column(const oam_model *m, int32_t b, int32_t a, int32_t k, float *d_out,
                                 void *stream) {
  if (!m || !d_out) return OAM_ERR_INVALID_ARG;
  if (b < -m->R || b > m->R || a < -m->R || a > m->R || k < 0 || k >= m->grid.nz) return OAM_ERR_INVALID_ARG;
  return slab_column(m, b, a, k, d_out, as_stream(stream));
}

oam_status oam_forward(const oam_model *m, const float *d_H, float *d_s, void *stream) {
  if (!m || !d_H || !d_s) return OAM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_H) | reinterpret_cast<uintptr_t>(d_s)) & 15) return OAM_ERR_INVALID_ARG;
  return apply_forward(m, d_H, d_s, as_stream(stream));
}

oam_status oam_adjoint(const oam_model *m, const float *d_s, float *d_H, void *stream) {
  if (!m || !d_H || !d_s) return OAM_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(d_H) | reinterpret_cast<uintptr_t>(d_s)) & 15) return OAM_ERR_INVALID_ARG;
  return apply_adjoint(m, d_s, d_H, as_stream(stream));
}

}  // extern "C"

// A filtered model (oam_model_set_filter) applies F A and A^T F.
oam_status oam::apply_forward(const oam_model *m, const float *H, float *s, cudaStream_t st) {
  oam_status rc;
  if (m->precision == OAM_PREC_BF16X3) rc = forward_tc(m, H, s, st);
  else if (m->precision == OAM_PREC_FFT) rc = forward_fft(m, H, s, st);
  else rc = forward_fp32(m, H, s, st);
  if (rc || !m->fir) return rc;
  return fir_apply(m, s, s, st);
}

oam_status oam::apply_adjoint(const oam_model *m, const float *s, float *H, cudaStream_t st) {
  if (m->fir) {
    float *fs = fir_stage(m);
    oam_status rc = fir_apply(m, s, fs, st);
    if (rc) return rc;
    s = fs;
  }
  if (m->precision == OAM_PREC_BF16X3) return adjoint_tc(m, s, H, st);
  if (m->precision == OAM_PREC_FFT) return adjoint_fft(m, s, H, st);
  return adjoint_fp32(m, s, H, st);
}
