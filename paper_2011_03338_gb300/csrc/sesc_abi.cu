// C ABI of the library (declared in include/sesc.h): handle, workspace,
// argument validation and the launch sequence of one right-hand side:
// K1 indicator + face states, K2 interface fluxes per direction, K3 update.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <new>
#include <vector>

#include "../../include/sesc.h"
#include "kparams.h"

using sesc::KParams;
using sesc::Work;

// launchers of the handle's precision
struct Launchers {
  int (*upload_ops)(int);
  int (*indicator)(const KParams&, const Work&, const double*, const double*, void*);
  int (*face_flux)(const KParams&, const Work&, void*);
  int (*update)(const KParams&, const Work&, const double*, const double*, double*, double, double, double,
                const double*, int, void*);
  int (*theta)(const KParams&, const Work&, double*, double*, void*);
  int (*dt)(const KParams&, const Work&, const double*, double*, void*);
  int (*update_x)(const KParams&, const Work&, const double*, const double*, double*, double, double, double,
                  const double*, const sesc::StageTerm&, void*);
  int (*stage_vjp)(const KParams&, const Work&, const double*, const double*, double, double, double, double*,
                   double*, double*, double*, void*);
  int (*pack_halo)(const KParams&, const Work&, int, int, void*, void*);
};

static const Launchers kFP64 = {sesc::fp64::upload_ops, sesc::fp64::launch_indicator, sesc::fp64::launch_face_flux,
                                sesc::fp64::launch_update, sesc::fp64::launch_theta, sesc::fp64::launch_dt,
                                sesc::fp64::launch_update_x, sesc::fp64::launch_stage_vjp,
                                sesc::fp64::launch_pack_halo};
static const Launchers kSplit = {sesc::split::upload_ops, sesc::split::launch_indicator,
                                 sesc::split::launch_face_flux, sesc::split::launch_update,
                                 sesc::split::launch_theta, sesc::split::launch_dt,
                                 sesc::split::launch_update_x, sesc::split::launch_stage_vjp,
                                 sesc::split::launch_pack_halo};

struct sesc_handle {
  sesc_config cfg;
  const Launchers* L;
  KParams kp;
  Work w;
  int device;
  int nl;
  size_t state_elems;   // E * nv * M^d
  double* stage[4];     // RK stage buffers (the last two allocated by the first SSP-RK(5,4) step)
  double* adj[2];       // adjoint scratch (element-face flux / state adjoints), allocated on first use
  int* classes;         // element-class lists: [16] counts, [16][E] lists
  // optional per-kernel timing: event pairs recorded around every launch
  bool timing;
  std::vector<cudaEvent_t> ev[SESC_NUM_KERNEL_KINDS][2];
};

namespace {

int ipow_i(int b, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

bool ops_ready[64][2][2];   // per device, precision and node family (guarded by ops_mu)
std::mutex ops_mu;

int validate(const sesc_config* c) {
  if (!c) return SESC_EINVAL;
  if (c->dim != 2 && c->dim != 3) return SESC_EINVAL;
  if (c->M != 4 && c->M != 8) return SESC_EINVAL;
  if (c->node_family != SESC_NODES_GAUSS && c->node_family != SESC_NODES_LOBATTO) return SESC_EINVAL;
  if (c->precision != SESC_FP64 && c->precision != SESC_FP32_SPLIT) return SESC_EINVAL;
  if (c->scheme != SESC_SCHEME_MULTI_LEVEL && c->scheme != SESC_SCHEME_SINGLE_LEVEL) return SESC_EINVAL;
  long long E = 1;
  for (int a = 0; a < c->dim; ++a) {
    if (c->nel[a] < 1) return SESC_EINVAL;
    if (!(c->xhi[a] > c->xlo[a])) return SESC_EINVAL;
    if (!(c->elem_size[a] >= 0.0) || c->elem_size[a] > 1e300) return SESC_EINVAL;
    const int lo = c->bc[2 * a], hi = c->bc[2 * a + 1];
    if (lo < 0 || lo > 3 || hi < 0 || hi > 3) return SESC_EINVAL;
    if ((lo == SESC_BC_PERIODIC) != (hi == SESC_BC_PERIODIC)) return SESC_EINVAL;
    E *= c->nel[a];
  }
  if (E > (1LL << 30)) return SESC_EINVAL;
  if (!(c->gamma > 1.0) || !(c->tauA > 0.0) || !(c->tauS >= 0.0) || !(c->cfl > 0.0)) return SESC_EINVAL;
  if (!(c->alphaL >= 0.0 && c->alphaH <= 1.0 && c->alphaL < c->alphaH)) return SESC_EINVAL;
  if (!(c->betaL >= 0.0 && c->betaL <= 1.0)) return SESC_EINVAL;
  return SESC_OK;
}

bool has_halo(const sesc_handle* h) {
  for (int i = 0; i < 2 * h->kp.dim; ++i)
    if (h->kp.bc[i] == SESC_BC_HALO) return true;
  return false;
}

// every halo side has its neighbour's face states set
bool halos_ready(const sesc_handle* h) {
  for (int i = 0; i < 2 * h->kp.dim; ++i)
    if (h->kp.bc[i] == SESC_BC_HALO && h->w.halo[i] == nullptr) return false;
  return true;
}

void free_work(sesc_handle* h) {
  cudaFree(h->w.face_states);
  cudaFree(h->w.face_flux);
  cudaFree(h->w.coeffs);
  cudaFree(h->w.decision);
  cudaFree(h->w.lmax);
  cudaFree(h->w.dt);
  cudaFree(h->w.counters);
  cudaFree(h->classes);
  for (int i = 0; i < 4; ++i) cudaFree(h->stage[i]);
  cudaFree(h->adj[0]);
  cudaFree(h->adj[1]);
}

int ensure_adjoint_scratch(sesc_handle* h) {
  if (h->adj[0]) return SESC_OK;
  const int d = h->kp.dim, nv = d + 2;
  int P = 1;
  for (int i = 0; i < d - 1; ++i) P *= h->kp.M;
  const size_t n = sizeof(double) * (size_t)h->kp.E * 2 * d * nv * P;
  if (cudaMalloc(&h->adj[0], n) != cudaSuccess || cudaMalloc(&h->adj[1], n) != cudaSuccess) {
    cudaFree(h->adj[0]);
    h->adj[0] = nullptr;
    cudaGetLastError();
    return SESC_ENOMEM;
  }
  return SESC_OK;
}

// NVTX range names of the launch kinds (seen by Nsight Systems / Compute timelines)
const char* const kRangeNames[SESC_NUM_KERNEL_KINDS] = {"sesc K1 indicator", "sesc K2 face flux",
                                                       "sesc K3 update", "sesc dt"};

// NVTX range and, with timing enabled, a pair of CUDA events around one launch group
struct Bracket {
  sesc_handle* h;
  int kind;
  cudaStream_t s;
  cudaEvent_t stop;
  Bracket(sesc_handle* hh, int k, void* stream) : h(hh), kind(k), s((cudaStream_t)stream), stop(nullptr) {
    nvtxRangePushA(kRangeNames[k]);
    if (!h->timing) return;
    cudaEvent_t start;
    if (cudaEventCreate(&start) != cudaSuccess || cudaEventCreate(&stop) != cudaSuccess) { stop = nullptr; return; }
    cudaEventRecord(start, s);
    h->ev[kind][0].push_back(start);
  }
  ~Bracket() {
    nvtxRangePop();
    if (!h->timing || !stop) return;
    cudaEventRecord(stop, s);
    h->ev[kind][1].push_back(stop);
  }
};

// one right-hand side evaluation into the update kernel (mode 0: dudt, 1: RK stage)
int run_rhs(sesc_handle* h, const double* us, const double* frozen, const double* u0, double* out, double a,
            double b, double dt, const double* dt_dev, int mode, void* stream) {
  if (!halos_ready(h)) return SESC_EINVAL;
  {
    Bracket br(h, SESC_KERNEL_INDICATOR, stream);
    if (h->L->indicator(h->kp, h->w, us, frozen, stream)) return SESC_ECUDA;
  }
  {
    Bracket br(h, SESC_KERNEL_FACE_FLUX, stream);
    if (h->L->face_flux(h->kp, h->w, stream)) return SESC_ECUDA;
  }
  {
    Bracket br(h, SESC_KERNEL_UPDATE, stream);
    if (h->L->update(h->kp, h->w, us, u0, out, a, b, dt, dt_dev, mode, stream)) return SESC_ECUDA;
  }
  return SESC_OK;
}

// one generalised RK stage (uout = a u0 + c u2 + b (us + g dt R(us)))
int run_stage_x(sesc_handle* h, const double* us, const double* u0, double* out, double a, double b, double dt,
                const double* dt_dev, const sesc::StageTerm& x, void* stream) {
  if (!halos_ready(h)) return SESC_EINVAL;
  {
    Bracket br(h, SESC_KERNEL_INDICATOR, stream);
    if (h->L->indicator(h->kp, h->w, us, nullptr, stream)) return SESC_ECUDA;
  }
  {
    Bracket br(h, SESC_KERNEL_FACE_FLUX, stream);
    if (h->L->face_flux(h->kp, h->w, stream)) return SESC_ECUDA;
  }
  Bracket br(h, SESC_KERNEL_UPDATE, stream);
  return h->L->update_x(h->kp, h->w, us, u0, out, a, b, dt, dt_dev, x, stream) ? SESC_ECUDA : SESC_OK;
}

int ensure_rk54_buffers(sesc_handle* h) {
  for (int i = 2; i < 4; ++i) {
    if (h->stage[i]) continue;
    if (cudaMalloc(&h->stage[i], sizeof(double) * h->state_elems) != cudaSuccess) {
      cudaGetLastError();
      return SESC_ENOMEM;
    }
  }
  return SESC_OK;
}

void clear_timing(sesc_handle* h) {
  for (int k = 0; k < SESC_NUM_KERNEL_KINDS; ++k)
    for (int j = 0; j < 2; ++j) {
      for (cudaEvent_t e : h->ev[k][j]) cudaEventDestroy(e);
      h->ev[k][j].clear();
    }
}

}  // namespace

namespace sesc {

// kernel parameters of a validated configuration
void make_params(const sesc_config* cfg, KParams* out, long long* nfaces_total) {
  const int d = cfg->dim, M = cfg->M;
  KParams& p = *out;
  p = KParams();
  p.stage_cap = kStageWaitCap;
  p.dim = d;
  p.M = M;
  long long E = 1;
  for (int a = 0; a < 3; ++a) p.nel[a] = (a < d) ? cfg->nel[a] : 1;
  for (int a = 0; a < d; ++a) E *= cfg->nel[a];
  p.E = (int)E;
  int S = 0;
  for (int n = M; n >= 2; n /= 2) S += ipow_i(M / n, d);
  p.S = S;
  for (int i = 0; i < 6; ++i) p.bc[i] = (i < 2 * d) ? cfg->bc[i] : 0;
  p.dxmin = 1e300;
  for (int a = 0; a < 3; ++a) {
    p.dx[a] = (a < d) ? (cfg->elem_size[a] > 0.0 ? cfg->elem_size[a] : (cfg->xhi[a] - cfg->xlo[a]) / cfg->nel[a])
                      : 1.0;
    p.mdx[a] = -(double)M / p.dx[a];
    if (a < d && p.dx[a] < p.dxmin) p.dxmin = p.dx[a];
  }
  p.gamma = cfg->gamma;
  p.tauA = cfg->tauA;
  p.tauS = cfg->tauS;
  p.alphaH = cfg->alphaH;
  p.alphaL = cfg->alphaL;
  p.betaL = cfg->betaL;
  p.cfl = cfg->cfl;
  p.family = cfg->node_family;
  p.single_level = cfg->scheme == SESC_SCHEME_SINGLE_LEVEL ? 1 : 0;
  p.fp32_filter = 1;
  long long nf_total = 0;
  for (int a = 0; a < 3; ++a) {
    p.face_off[a] = (int)nf_total;
    if (a >= d) { p.nfaces_along[a] = 0; continue; }
    p.nfaces_along[a] = (cfg->bc[2 * a] == SESC_BC_PERIODIC) ? cfg->nel[a] : cfg->nel[a] + 1;
    long long nf = p.nfaces_along[a];
    for (int b = 0; b < d; ++b)
      if (b != a) nf *= cfg->nel[b];
    nf_total += nf;
  }
  *nfaces_total = nf_total;
  p.nfaces = nf_total;
}

int validate_config(const sesc_config* cfg) { return validate(cfg); }

}  // namespace sesc

extern "C" {

int sesc_create(const sesc_config* cfg, sesc_handle** out) {
  if (!out) return SESC_EINVAL;
  *out = nullptr;
  int rc = validate(cfg);
  if (rc != SESC_OK) return rc;
  sesc_handle* h = new (std::nothrow) sesc_handle();
  if (!h) return SESC_ENOMEM;
  h->cfg = *cfg;
  h->L = (cfg->precision == SESC_FP32_SPLIT) ? &kSplit : &kFP64;
  if (cudaGetDevice(&h->device) != cudaSuccess) { delete h; return SESC_ECUDA; }
  const int d = cfg->dim, M = cfg->M;
  KParams& p = h->kp;
  long long nfaces_total = 0;
  sesc::make_params(cfg, &p, &nfaces_total);
  const long long E = p.E;
  const int S = p.S;
  const int nv = d + 2;
  const int MD = ipow_i(M, d), P = ipow_i(M, d - 1);
  int nl = 1;
  for (int n = M; n >= 2; n /= 2) ++nl;
  h->nl = nl;
  h->state_elems = (size_t)E * nv * MD;
  if (h->device < 0 || h->device >= 64) { delete h; return SESC_EINVAL; }
  const int pi = (cfg->precision == SESC_FP32_SPLIT) ? 1 : 0;
  {
    std::lock_guard<std::mutex> lock(ops_mu);
    if (!ops_ready[h->device][pi][p.family]) {
      if (h->L->upload_ops(p.family) != 0) { delete h; return SESC_ECUDA; }
      ops_ready[h->device][pi][p.family] = true;
    }
  }
  bool ok = true;
  ok = ok && cudaMalloc(&h->w.face_states, sizeof(double) * (size_t)E * 2 * d * (nv + nl) * P) == cudaSuccess;
  ok = ok && cudaMalloc(&h->w.face_flux, sizeof(double) * (size_t)nfaces_total * nv * P) == cudaSuccess;
  ok = ok && cudaMalloc(&h->w.coeffs, sizeof(double) * (size_t)E * 2 * S) == cudaSuccess;
  ok = ok && cudaMalloc(&h->w.decision, (size_t)E) == cudaSuccess;
  ok = ok && cudaMalloc(&h->w.lmax, 2 * sizeof(unsigned long long)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->w.dt, sizeof(double)) == cudaSuccess;
  ok = ok && cudaMalloc(&h->w.counters, sizeof(long long) * sesc::kCounters) == cudaSuccess;
  ok = ok && cudaMalloc(&h->stage[0], sizeof(double) * h->state_elems) == cudaSuccess;
  ok = ok && cudaMalloc(&h->stage[1], sizeof(double) * h->state_elems) == cudaSuccess;
  // the update kernel takes its elements class by class when several CTAs share an SM
  // (at least 4) over many waves (at least 8 times the CTAs resident at once): measured
  // 7 % faster on the 2D M = 8 256^2 workload in FP32 (1.4 % in FP64); up to 6 % slower
  // on meshes of a few waves (every CTA waits for the lists at start) and 4 % slower in
  // 3D M = 8 (one or two 512-thread CTAs per SM)
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
  const int per_sm = (cfg->precision == SESC_FP32_SPLIT) ? sesc::split::batch_max_blocks(d, M, 2)
                                                         : sesc::fp64::batch_max_blocks(d, M, 2);
  if (ok && per_sm >= 4 && E >= 8LL * sms * per_sm) {
    ok = cudaMalloc(&h->classes, sizeof(int) * (16 + 17 * (size_t)E)) == cudaSuccess;
    ok = ok && cudaMemset(h->classes, 0, sizeof(int) * 16) == cudaSuccess;
    if (ok) {
      h->w.class_count = h->classes;
      h->w.class_list = h->classes + 16;
      // FP32 build: K1 follows the order K3 took last (K1 2.5 % faster on the 2D M = 8
      // 256^2 workload; in FP64 0.5 % slower, so FP64 handles keep the mesh order there)
      if (cfg->precision == SESC_FP32_SPLIT) {
        h->w.order = h->classes + 16 + 16 * (size_t)E;
        std::vector<int> iota((size_t)E);
        for (long long i = 0; i < E; ++i) iota[(size_t)i] = (int)i;
        ok = cudaMemcpy(h->w.order, iota.data(), sizeof(int) * (size_t)E, cudaMemcpyHostToDevice) == cudaSuccess;
      }
    }
  }
  if (!ok) {
    free_work(h);
    delete h;
    cudaGetLastError();
    return SESC_ENOMEM;
  }
  if (cudaMemset(h->w.counters, 0, sizeof(long long) * sesc::kCounters) != cudaSuccess) {
    free_work(h);
    delete h;
    return SESC_ECUDA;
  }
  *out = h;
  return SESC_OK;
}

void sesc_destroy(sesc_handle* h) {
  if (!h) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  clear_timing(h);
  free_work(h);
  cudaSetDevice(prev);
  delete h;
}

int64_t sesc_num_elements(const sesc_handle* h) { return h ? (int64_t)h->kp.E : -1; }
int64_t sesc_num_coeffs(const sesc_handle* h) { return h ? (int64_t)h->kp.S : -1; }

int sesc_indicator(sesc_handle* h, const double* u, double* coeffs, double* theta, uint8_t* decision, double* abar,
                   void* stream) {
  if (!h || !u) return SESC_EINVAL;
  if (h->L->indicator(h->kp, h->w, u, nullptr, stream)) return SESC_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  if (coeffs && cudaMemcpyAsync(coeffs, h->w.coeffs, sizeof(double) * (size_t)h->kp.E * 2 * h->kp.S,
                                cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return SESC_ECUDA;
  if (decision && cudaMemcpyAsync(decision, h->w.decision, (size_t)h->kp.E, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return SESC_ECUDA;
  if ((theta || abar) && h->L->theta(h->kp, h->w, theta, abar, stream)) return SESC_ECUDA;
  return SESC_OK;
}

int sesc_rhs(sesc_handle* h, const double* u, double* dudt, const double* frozen, double* coeffs_out, void* stream) {
  if (!h || !u || !dudt || u == dudt) return SESC_EINVAL;
  int rc = run_rhs(h, u, frozen, nullptr, dudt, 0.0, 1.0, 0.0, nullptr, 0, stream);
  if (rc != SESC_OK) return rc;
  if (coeffs_out && cudaMemcpyAsync(coeffs_out, h->w.coeffs, sizeof(double) * (size_t)h->kp.E * 2 * h->kp.S,
                                    cudaMemcpyDeviceToDevice, (cudaStream_t)stream) != cudaSuccess)
    return SESC_ECUDA;
  return SESC_OK;
}

int sesc_rk_stage(sesc_handle* h, const double* u0, const double* us, double* uout, double a, double b, double dt,
                  const double* dt_dev, const double* frozen, double* coeffs_out, void* stream) {
  if (!h || !us || !uout || uout == us) return SESC_EINVAL;
  if (a != 0.0 && !u0) return SESC_EINVAL;
  int rc = run_rhs(h, us, frozen, u0, uout, a, b, dt, dt_dev, 1, stream);
  if (rc != SESC_OK) return rc;
  if (coeffs_out && cudaMemcpyAsync(coeffs_out, h->w.coeffs, sizeof(double) * (size_t)h->kp.E * 2 * h->kp.S,
                                    cudaMemcpyDeviceToDevice, (cudaStream_t)stream) != cudaSuccess)
    return SESC_ECUDA;
  return SESC_OK;
}

int sesc_dt(sesc_handle* h, const double* u, double* dt_dev, void* stream) {
  if (!h || !u) return SESC_EINVAL;
  Bracket br(h, SESC_KERNEL_DT, stream);
  return h->L->dt(h->kp, h->w, u, dt_dev, stream) ? SESC_ECUDA : SESC_OK;
}

int sesc_rk3_step(sesc_handle* h, const double* u, double* uout, double* dt_dev, void* stream) {
  if (!h || !u || !uout) return SESC_EINVAL;
  {
    Bracket br(h, SESC_KERNEL_DT, stream);
    if (h->L->dt(h->kp, h->w, u, dt_dev, stream)) return SESC_ECUDA;
  }
  const double* dtp = h->w.dt;
  int rc = run_rhs(h, u, nullptr, u, h->stage[0], 0.0, 1.0, 0.0, dtp, 1, stream);
  if (rc == SESC_OK) rc = run_rhs(h, h->stage[0], nullptr, u, h->stage[1], 0.75, 0.25, 0.0, dtp, 1, stream);
  if (rc == SESC_OK) rc = run_rhs(h, h->stage[1], nullptr, u, uout, 1.0 / 3.0, 2.0 / 3.0, 0.0, dtp, 1, stream);
  return rc;
}

int sesc_rk_stage_ex(sesc_handle* h, const double* u0, double a, const double* u2, double c, const double* us,
                     double b, double g, double dt, const double* dt_dev, double* uout, void* stream) {
  if (!h || !us || !uout || uout == us) return SESC_EINVAL;
  if ((a != 0.0 && !u0) || (c != 0.0 && !u2)) return SESC_EINVAL;
  const sesc::StageTerm x{c != 0.0 ? u2 : nullptr, c, g};
  return run_stage_x(h, us, a != 0.0 ? u0 : us, uout, a, b, dt, dt_dev, x, stream);
}

int sesc_ssprk54_step(sesc_handle* h, const double* u, double* uout, double* dt_dev, void* stream) {
  if (!h || !u || !uout) return SESC_EINVAL;
  int rc = ensure_rk54_buffers(h);
  if (rc != SESC_OK) return rc;
  {
    Bracket br(h, SESC_KERNEL_DT, stream);
    if (h->L->dt(h->kp, h->w, u, dt_dev, stream)) return SESC_ECUDA;
  }
  // Shu-Osher coefficients of SSP-RK(5,4) (Spiteri & Ruuth 2002):
  //   u1 = u + b10 dt L(u)
  //   u2 = a20 u + a21 u1 + b21 dt L(u1)
  //   u3 = a30 u + a32 u2 + b32 dt L(u2)
  //   u4 = a40 u + a43 u3 + b43 dt L(u3)
  //   u5 = a52 u2 + a53 u3 + b53 dt L(u3) + a54 u4 + b54 dt L(u4)
  // a53 / a43 = b53 / b43 (= k), so a53 u3 + b53 dt L(u3) = k (u4 - a40 u) and the
  // last stage needs L(u4) only: u5 = -k a40 u + a52 u2 + (a54 + k) u4 + b54 dt L(u4).
  const double b10 = 0.391752226571890;
  const double a20 = 0.444370493651235, a21 = 0.555629506348765, b21 = 0.368410593050371;
  const double a30 = 0.620101851488403, a32 = 0.379898148511597, b32 = 0.251891774271694;
  const double a40 = 0.178079954393132, a43 = 0.821920045606868, b43 = 0.544974750228521;
  const double a52 = 0.517231671970585, a53 = 0.096059710526147, a54 = 0.386708617503269;
  const double b54 = 0.226007483236906;
  const double k = a53 / a43;
  const double* dtp = h->w.dt;
  double* s1 = h->stage[0];
  double* s2 = h->stage[1];
  double* s3 = h->stage[2];
  double* s4 = h->stage[3];
  rc = run_stage_x(h, u, u, s1, 0.0, 1.0, 0.0, dtp, sesc::StageTerm{nullptr, 0.0, b10}, stream);
  if (rc == SESC_OK) rc = run_stage_x(h, s1, u, s2, a20, a21, 0.0, dtp, sesc::StageTerm{nullptr, 0.0, b21 / a21}, stream);
  if (rc == SESC_OK) rc = run_stage_x(h, s2, u, s3, a30, a32, 0.0, dtp, sesc::StageTerm{nullptr, 0.0, b32 / a32}, stream);
  if (rc == SESC_OK) rc = run_stage_x(h, s3, u, s4, a40, a43, 0.0, dtp, sesc::StageTerm{nullptr, 0.0, b43 / a43}, stream);
  if (rc == SESC_OK)
    rc = run_stage_x(h, s4, u, uout, -k * a40, a54 + k, 0.0, dtp, sesc::StageTerm{s2, a52, b54 / (a54 + k)}, stream);
  return rc;
}

int64_t sesc_halo_bytes(const sesc_handle* h, int side) {
  if (!h || side < 0 || side >= 2 * h->kp.dim) return -1;
  const int d = h->kp.dim, a = side / 2;
  long long ntr = 1;
  for (int b = 0; b < d; ++b)
    if (b != a) ntr *= h->kp.nel[b];
  const int P = ipow_i(h->kp.M, d - 1);
  const size_t esz = (h->cfg.precision == SESC_FP32_SPLIT) ? sizeof(float) : sizeof(double);
  return (int64_t)(ntr * (d + 2 + h->nl) * P * (long long)esz);
}

int sesc_pack_halo(sesc_handle* h, int side, void* dst, void* stream) {
  if (!h || !dst || side < 0 || side >= 2 * h->kp.dim) return SESC_EINVAL;
  return h->L->pack_halo(h->kp, h->w, side / 2, side % 2, dst, stream) ? SESC_ECUDA : SESC_OK;
}

int sesc_set_halo(sesc_handle* h, int side, const void* src) {
  if (!h || side < 0 || side >= 2 * h->kp.dim || h->kp.bc[side] != SESC_BC_HALO) return SESC_EINVAL;
  h->w.halo[side] = src;
  return SESC_OK;
}

int sesc_stage_finish(sesc_handle* h, const double* u0, const double* us, double* out, double a, double b, double dt,
                      const double* dt_dev, int mode, void* stream) {
  if (!h || !us || !out || out == us || (mode != 0 && mode != 1)) return SESC_EINVAL;
  if (mode == 1 && a != 0.0 && !u0) return SESC_EINVAL;
  if (!halos_ready(h)) return SESC_EINVAL;
  {
    Bracket br(h, SESC_KERNEL_FACE_FLUX, stream);
    if (h->L->face_flux(h->kp, h->w, stream)) return SESC_ECUDA;
  }
  Bracket br(h, SESC_KERNEL_UPDATE, stream);
  return h->L->update(h->kp, h->w, us, mode ? u0 : nullptr, out, a, b, dt, dt_dev, mode, stream) ? SESC_ECUDA
                                                                                                 : SESC_OK;
}

int sesc_status(sesc_handle* h, int64_t* counters) {
  if (!h) return SESC_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  long long c[16];
  cudaError_t e1 = cudaDeviceSynchronize();
  cudaError_t e2 = cudaMemcpy(c, h->w.counters, sizeof(c), cudaMemcpyDeviceToHost);
  cudaSetDevice(prev);
  if (e1 != cudaSuccess || e2 != cudaSuccess) return SESC_ECUDA;
  if (counters)
    for (int i = 0; i < 16; ++i) counters[i] = (int64_t)c[i];
  if (c[0] & 8) return SESC_EBOUNDS;
  if (c[0] & 4) return SESC_ETIMEOUT;
  if (c[0] & 1) return SESC_ENONPERMISSIBLE;
  if (c[0] & 2) return SESC_ENONFINITE;
  return SESC_OK;
}

int sesc_level_counts(sesc_handle* h, int64_t* counts) {
  if (!h || !counts) return SESC_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  long long c[sesc::kCounters];
  cudaError_t e1 = cudaDeviceSynchronize();
  cudaError_t e2 = cudaMemcpy(c, h->w.counters, sizeof(c), cudaMemcpyDeviceToHost);
  cudaSetDevice(prev);
  if (e1 != cudaSuccess || e2 != cudaSuccess) return SESC_ECUDA;
  for (int m = 0; m < 16; ++m) counts[m] = (int64_t)c[16 + m];
  return SESC_OK;
}

int sesc_set_stage_cap(sesc_handle* h, int64_t polls) {
  if (!h || polls < 0) return SESC_EINVAL;
  h->kp.stage_cap = (long long)polls;
  return SESC_OK;
}

int sesc_set_indicator_filter(sesc_handle* h, int on) {
  if (!h) return SESC_EINVAL;
  h->kp.fp32_filter = on ? 1 : 0;
  return SESC_OK;
}

int sesc_reset_status(sesc_handle* h, void* stream) {
  if (!h) return SESC_EINVAL;
  return cudaMemsetAsync(h->w.counters, 0, sizeof(long long) * sesc::kCounters, (cudaStream_t)stream) == cudaSuccess ? SESC_OK
                                                                                                       : SESC_ECUDA;
}

int sesc_rk_stage_vjp(sesc_handle* h, const double* us, const double* frozen, const double* uout_bar, double a,
                      double b, double dt, const double* dt_dev, double* us_bar, double* u0_bar, void* stream) {
  if (!h || !us || !uout_bar || !us_bar) return SESC_EINVAL;
  if (h->cfg.scheme != SESC_SCHEME_MULTI_LEVEL || has_halo(h)) return SESC_EINVAL;
  if (dt_dev) {
    // the scale b dt is needed on the host: one synchronous read of the device time step
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return SESC_ECUDA;
    if (cudaMemcpy(&dt, dt_dev, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess) return SESC_ECUDA;
  }
  int rc = ensure_adjoint_scratch(h);
  if (rc != SESC_OK) return rc;
  {
    Bracket br(h, SESC_KERNEL_INDICATOR, stream);
    if (h->L->indicator(h->kp, h->w, us, frozen, stream)) return SESC_ECUDA;
  }
  Bracket br(h, SESC_KERNEL_UPDATE, stream);
  if (h->L->stage_vjp(h->kp, h->w, us, uout_bar, a, b, b * dt, us_bar, u0_bar, h->adj[0], h->adj[1], stream))
    return SESC_ECUDA;
  return SESC_OK;
}

int sesc_rhs_vjp(sesc_handle* h, const double* u, const double* frozen, const double* dudt_bar, double* u_bar,
                 void* stream) {
  if (!h || !u || !dudt_bar || !u_bar) return SESC_EINVAL;
  if (h->cfg.scheme != SESC_SCHEME_MULTI_LEVEL || has_halo(h)) return SESC_EINVAL;
  int rc = ensure_adjoint_scratch(h);
  if (rc != SESC_OK) return rc;
  if (cudaMemsetAsync(u_bar, 0, sizeof(double) * h->state_elems, (cudaStream_t)stream) != cudaSuccess)
    return SESC_ECUDA;
  if (h->L->indicator(h->kp, h->w, u, frozen, stream)) return SESC_ECUDA;
  if (h->L->stage_vjp(h->kp, h->w, u, dudt_bar, 0.0, 0.0, 1.0, u_bar, nullptr, h->adj[0], h->adj[1], stream))
    return SESC_ECUDA;
  return SESC_OK;
}

int sesc_set_timing(sesc_handle* h, int enable) {
  if (!h) return SESC_EINVAL;
  h->timing = enable != 0;
  return SESC_OK;
}

int sesc_kernel_times(sesc_handle* h, double* ms, int64_t* launches) {
  if (!h || !ms || !launches) return SESC_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  cudaError_t err = cudaDeviceSynchronize();
  int rc = (err == cudaSuccess) ? SESC_OK : SESC_ECUDA;
  for (int k = 0; k < SESC_NUM_KERNEL_KINDS; ++k) {
    double total = 0.0;
    const size_t n = h->ev[k][1].size();
    for (size_t i = 0; i < n; ++i) {
      float t = 0.0f;
      if (cudaEventElapsedTime(&t, h->ev[k][0][i], h->ev[k][1][i]) == cudaSuccess) total += t;
      else rc = SESC_ECUDA;
    }
    ms[k] = total;
    launches[k] = (int64_t)n;
  }
  clear_timing(h);
  cudaSetDevice(prev);
  return rc;
}

const char* sesc_strerror(int code) {
  switch (code) {
    case SESC_OK: return "ok";
    case SESC_EINVAL: return "invalid argument or configuration";
    case SESC_ENOMEM: return "device allocation failed";
    case SESC_ECUDA: return "CUDA call or kernel launch failed";
    case SESC_ENONPERMISSIBLE: return "a mean value is not permissible (rho <= 0 or p <= 0)";
    case SESC_ENONFINITE: return "non-finite wave speed in the time-step reduction";
    case SESC_ETOOLARGE: return "problem too large for the static scratch of sesc_rhs_static";
    case SESC_EBOUNDS: return "a computed index fell outside its buffer (bounds-checked build)";
    case SESC_ETIMEOUT: return "a bounded device-side wait (grid barrier or staging copy) timed out";
    default: return "unknown error";
  }
}

}  // extern "C"
