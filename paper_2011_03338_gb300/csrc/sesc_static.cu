// sesc_rhs_static: the right-hand side without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: applications that hand out
// a fixed device-memory budget up front and forbid allocations behind their
// back (a host simulation code, a plugin inside another program), and callers
// on a time-critical path, where cudaMalloc / cudaFree can synchronise the
// device and stall work on other streams. For them this entry point runs the
// same three kernels as sesc_rhs, with the scratch (face states, interface
// fluxes, coefficients, decisions, counters) carved out of one file-scope
// device array instead of a handle's workspace.
//
// The array below is a host-side stand-in in host code: its device address is
// obtained once per device with cudaGetSymbolAddress and passed to the kernels.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sesc.h"
#include "kparams.h"

// The scratch shared by every call on a device (SESC_STATIC_SCRATCH_BYTES).
static __device__ __align__(256) unsigned char g_scratch[SESC_STATIC_SCRATCH_BYTES];

namespace {

struct DeviceSetup {
  bool ready;
  bool ops[2];
  unsigned char* scratch;   // device address of g_scratch on this device
};
DeviceSetup g_setup[64];

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int ipow_s(int b, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// configuration checks and kernel parameters (same rules as sesc_create)
int params_of(const sesc_config* c, sesc::KParams* p, size_t* nfaces_total) {
  if (!c) return SESC_EINVAL;
  if (c->dim != 2 && c->dim != 3) return SESC_EINVAL;
  if (c->M != 4 && c->M != 8) return SESC_EINVAL;
  if (c->node_family != SESC_NODES_GAUSS && c->node_family != SESC_NODES_LOBATTO) return SESC_EINVAL;
  if (c->precision != SESC_FP64) return SESC_EINVAL;
  if (c->scheme != SESC_SCHEME_MULTI_LEVEL && c->scheme != SESC_SCHEME_SINGLE_LEVEL) return SESC_EINVAL;
  if (!(c->gamma > 1.0) || !(c->tauA > 0.0) || !(c->tauS >= 0.0) || !(c->cfl > 0.0)) return SESC_EINVAL;
  if (!(c->alphaL >= 0.0 && c->alphaH <= 1.0 && c->alphaL < c->alphaH)) return SESC_EINVAL;
  if (!(c->betaL >= 0.0 && c->betaL <= 1.0)) return SESC_EINVAL;
  const int d = c->dim, M = c->M;
  long long E = 1;
  for (int a = 0; a < d; ++a) {
    if (c->nel[a] < 1 || !(c->xhi[a] > c->xlo[a])) return SESC_EINVAL;
    const int lo = c->bc[2 * a], hi = c->bc[2 * a + 1];
    if (lo < 0 || lo > 2 || hi < 0 || hi > 2) return SESC_EINVAL;
    if ((lo == SESC_BC_PERIODIC) != (hi == SESC_BC_PERIODIC)) return SESC_EINVAL;
    E *= c->nel[a];
    if (E > (1LL << 30)) return SESC_ETOOLARGE;
  }
  *p = sesc::KParams();
  p->dim = d;
  p->M = M;
  p->E = (int)E;
  int S = 0;
  for (int n = M; n >= 2; n /= 2) S += ipow_s(M / n, d);
  p->S = S;
  for (int a = 0; a < 3; ++a) p->nel[a] = (a < d) ? c->nel[a] : 1;
  for (int i = 0; i < 6; ++i) p->bc[i] = (i < 2 * d) ? c->bc[i] : 0;
  p->dxmin = 1e300;
  for (int a = 0; a < 3; ++a) {
    p->dx[a] = (a < d) ? (c->xhi[a] - c->xlo[a]) / c->nel[a] : 1.0;
    p->mdx[a] = -(double)M / p->dx[a];
    if (a < d && p->dx[a] < p->dxmin) p->dxmin = p->dx[a];
  }
  p->gamma = c->gamma;
  p->tauA = c->tauA;
  p->tauS = c->tauS;
  p->alphaH = c->alphaH;
  p->alphaL = c->alphaL;
  p->betaL = c->betaL;
  p->cfl = c->cfl;
  p->family = c->node_family;
  p->single_level = c->scheme == SESC_SCHEME_SINGLE_LEVEL ? 1 : 0;
  size_t nf_total = 0;
  for (int a = 0; a < 3; ++a) {
    p->face_off[a] = (int)nf_total;
    if (a >= d) { p->nfaces_along[a] = 0; continue; }
    p->nfaces_along[a] = (c->bc[2 * a] == SESC_BC_PERIODIC) ? c->nel[a] : c->nel[a] + 1;
    size_t nf = (size_t)p->nfaces_along[a];
    for (int b = 0; b < d; ++b)
      if (b != a) nf *= (size_t)c->nel[b];
    nf_total += nf;
  }
  *nfaces_total = nf_total;
  return SESC_OK;
}

}  // namespace

extern "C" int sesc_rhs_static(const sesc_config* cfg, const double* u, double* dudt, void* stream) {
  if (!u || !dudt || u == dudt) return SESC_EINVAL;
  sesc::KParams p;
  size_t nfaces = 0;
  int rc = params_of(cfg, &p, &nfaces);
  if (rc != SESC_OK) return rc;
  const int d = p.dim, M = p.M, nv = d + 2;
  const size_t P = (size_t)ipow_s(M, d - 1);
  int nl = 1;
  for (int n = M; n >= 2; n /= 2) ++nl;
  // scratch layout, every block 256-byte aligned
  const size_t b_fs = align256(sizeof(double) * (size_t)p.E * 2 * d * (nv + nl) * P);
  const size_t b_ff = align256(sizeof(double) * nfaces * nv * P);
  const size_t b_co = align256(sizeof(double) * (size_t)p.E * 2 * p.S);
  const size_t b_de = align256((size_t)p.E);
  const size_t b_lm = 256, b_dt = 256, b_ct = align256(sizeof(long long) * 16);
  const size_t total = b_fs + b_ff + b_co + b_de + b_lm + b_dt + b_ct;
  if (total > (size_t)SESC_STATIC_SCRATCH_BYTES) return SESC_ETOOLARGE;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SESC_ECUDA;
  if (dev < 0 || dev >= 64) return SESC_EINVAL;
  DeviceSetup& st = g_setup[dev];
  if (!st.ready) {
    void* addr = nullptr;
    if (cudaGetSymbolAddress(&addr, g_scratch) != cudaSuccess || addr == nullptr) return SESC_ECUDA;
    st.scratch = static_cast<unsigned char*>(addr);
    st.ready = true;
  }
  if (!st.ops[p.family]) {
    if (sesc::fp64::upload_ops(p.family) != 0) return SESC_ECUDA;
    st.ops[p.family] = true;
  }
  unsigned char* base = st.scratch;
  sesc::Work w;
  w.face_states = reinterpret_cast<double*>(base);
  base += b_fs;
  w.face_flux = reinterpret_cast<double*>(base);
  base += b_ff;
  w.coeffs = reinterpret_cast<double*>(base);
  base += b_co;
  w.decision = base;
  base += b_de;
  w.lmax = reinterpret_cast<unsigned long long*>(base);
  base += b_lm;
  w.dt = reinterpret_cast<double*>(base);
  base += b_dt;
  w.counters = reinterpret_cast<long long*>(base);
  // the array keeps the previous call's contents: counters must start at zero
  if (cudaMemsetAsync(w.counters, 0, sizeof(long long) * 16, (cudaStream_t)stream) != cudaSuccess) return SESC_ECUDA;
  if (sesc::fp64::launch_indicator(p, w, u, nullptr, stream)) return SESC_ECUDA;
  if (sesc::fp64::launch_face_flux(p, w, stream)) return SESC_ECUDA;
  if (sesc::fp64::launch_update(p, w, u, nullptr, dudt, 0.0, 1.0, 0.0, nullptr, 0, stream)) return SESC_ECUDA;
  return SESC_OK;
}
