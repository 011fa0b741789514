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
// Where the scratch lives: g_scratch below is a device array (one copy in the
// memory of every GPU that loads the library). In host code its name refers to a
// host-side shadow of that array, not to device memory, so host code never hands
// &g_scratch to a kernel: the device address of this device's copy is looked up
// once per device with cudaGetSymbolAddress and the kernels get that pointer.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>

#include "../../include/sesc.h"
#include "kparams.h"

// The scratch shared by every call on a device (SESC_STATIC_SCRATCH_BYTES).
static __device__ __align__(256) unsigned char g_scratch[SESC_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;

// Per-device set-up: the device address of g_scratch and the operator tables of
// each node family. Done under a mutex, so host threads that make their first
// calls on a device at the same time do not race on it; afterwards the flags are
// read without the lock.
struct DeviceSetup {
  std::atomic<bool> ready{false};
  std::atomic<bool> ops[2] = {false, false};
  unsigned char* scratch = nullptr;   // device address of g_scratch on this device
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mu;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int ipow_s(int b, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// device address of this device's scratch and its operator tables for `family`
int device_setup(int dev, int family, unsigned char** scratch) {
  DeviceSetup& st = g_setup[dev];
  if (!st.ready.load(std::memory_order_acquire) || !st.ops[family].load(std::memory_order_acquire)) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!st.ready.load(std::memory_order_relaxed)) {
      void* addr = nullptr;
      if (cudaGetSymbolAddress(&addr, g_scratch) != cudaSuccess || addr == nullptr) return SESC_ECUDA;
      st.scratch = static_cast<unsigned char*>(addr);
      st.ready.store(true, std::memory_order_release);
    }
    if (!st.ops[family].load(std::memory_order_relaxed)) {
      if (sesc::fp64::upload_ops(family) != 0) return SESC_ECUDA;
      st.ops[family].store(true, std::memory_order_release);
    }
  }
  *scratch = st.scratch;
  return SESC_OK;
}

}  // namespace

extern "C" int sesc_rhs_static(const sesc_config* cfg, const double* u, double* dudt, void* stream) {
  if (!u || !dudt || u == dudt) return SESC_EINVAL;
  // same configuration rules and kernel parameters as sesc_create
  int rc = sesc::validate_config(cfg);
  if (rc != SESC_OK) return rc;
  if (cfg->precision != SESC_FP64) return SESC_EINVAL;
  for (int i = 0; i < 2 * cfg->dim; ++i)
    if (cfg->bc[i] == SESC_BC_HALO) return SESC_EINVAL;   // no way to pass a neighbour's face states
  sesc::KParams p;
  long long nfaces_ll = 0;
  sesc::make_params(cfg, &p, &nfaces_ll);
  const size_t nfaces = (size_t)nfaces_ll;
  const int d = p.dim, M = p.M, nv = d + 2;
  const size_t P = (size_t)ipow_s(M, d - 1);
  int nl = 1;
  for (int n = M; n >= 2; n /= 2) ++nl;
  // scratch layout, every block 256-byte aligned
  const size_t b_fs = align256(sizeof(double) * (size_t)p.E * 2 * d * (nv + nl) * P);
  const size_t b_ff = align256(sizeof(double) * nfaces * nv * P);
  const size_t b_co = align256(sizeof(double) * (size_t)p.E * 2 * p.S);
  const size_t b_de = align256((size_t)p.E);
  const size_t b_lm = 256, b_dt = 256, b_ct = align256(sizeof(long long) * sesc::kCounters);
  const size_t total = b_fs + b_ff + b_co + b_de + b_lm + b_dt + b_ct;
  if (total > (size_t)SESC_STATIC_SCRATCH_BYTES) return SESC_ETOOLARGE;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SESC_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return SESC_EINVAL;
  unsigned char* base = nullptr;
  rc = device_setup(dev, p.family, &base);
  if (rc != SESC_OK) return rc;
  sesc::Work w{};
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
  if (cudaMemsetAsync(w.counters, 0, sizeof(long long) * sesc::kCounters, (cudaStream_t)stream) != cudaSuccess)
    return SESC_ECUDA;
  if (sesc::fp64::launch_indicator(p, w, u, nullptr, stream)) return SESC_ECUDA;
  if (sesc::fp64::launch_face_flux(p, w, stream)) return SESC_ECUDA;
  if (sesc::fp64::launch_update(p, w, u, nullptr, dudt, 0.0, 1.0, 0.0, nullptr, 0, stream)) return SESC_ECUDA;
  return SESC_OK;
}
