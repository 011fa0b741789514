// Kernels of the multi-level blended DG/FV right-hand side, written once for a
// compute type `real` (included by kernels_fp64.cu with real = double and by
// kernels_split.cu with real = float; the including file defines SESC_REAL and
// SESC_NS before the include).
//
// K1 k_indicator  per level: reconstruction (eqs. reco-2nd-order ... reco-8th-order,
//                 3D-nodal-reconstruction), squeezing beta (eq. calc-squeezing-
//                 parameter, two-step reading), smoothness sigma (eq. L1-norm-slope)
//                 and blending factor (eq. calc-blending-factor); the high-to-low
//                 snapping loop of the multi-level sketch; blending weights theta
//                 (eq. blending-weights); blended face-centred states of the 2d
//                 element faces (eq. 3D-prolongation for every level).
// K2 k_face_flux  common interface flux at element faces: F^(1) = f*(Ubar_L, Ubar_R)
//                 and level-n candidates P f*(R Ubar R^T) P^T (eqs. 3D-boundary-
//                 value-recon ... 3D-blend-interface-fluxes), weights (theta_L +
//                 theta_R) / 2.
// K3 k_update     inner interface fluxes; every active level's right-hand side in
//                 subcell-flux (telescoping) form: interior fluxes G from the
//                 cumulative volume operator, the common fluxes at sub-element
//                 boundaries (eqs. multilevel-blending-scheme, dgfv-scheme-3d); the
//                 theta blend of the flux differences, accumulated in FP64; the RK
//                 stage in FP64.
// k_lambda/k_dt   time step of eq. cfl-condition (FP64).
//
// FP64 islands whatever `real` is: the indicator ratio and blending factor, the
// squeezing formula, the permissibility checks of blended / reconstructed face
// states (division-free: rho > 0 and 2 rho E > |m|^2), the assembly of the flux
// differences and the RK stage. With real = float everything else (reconstruction,
// nodal and interface fluxes, operator passes) runs in FP32.

namespace sesc {
namespace SESC_NS {

typedef SESC_REAL real;

// ---------------------------------------------------------------------------
// operator tables in constant memory: [node family][log2 n]
// ---------------------------------------------------------------------------
struct DevLevel {
  real R[64], P[64], Dn[64], C[64], IRf[72], c0[8], cn[8], w[8];
  real lamR, lamI;   // largest absolute row sums of R and of I R (bounds of the point values)
};
struct DevOps {
  DevLevel lv[3];   // levels n = 2, 4, 8 (lv[log2 n - 1])
};
static __constant__ DevOps c_ops[2];

// FP32 copies of the tables that the certified FP32 pass of the FP64 indicator uses
// (indicator_f32): [node family][log2 n - 1]
struct DevLevelF {
  float R[64], Dn[64], Dna[64], IRf[72], w[8];   // Dna = |Dn| entrywise
  float lamR, lamI;                              // largest absolute row sums of R and of IRf, rounded up
};
static __constant__ DevLevelF c_opsf[2][3];

// ---------------------------------------------------------------------------
// compile-time geometry
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }
__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
__host__ __device__ constexpr int cpopc(int x) { return x == 0 ? 0 : (x & 1) + cpopc(x >> 1); }
__host__ __device__ constexpr int s_total(int M, int D, int n) { return n < 2 ? 0 : ipow(M / n, D) + s_total(M, D, n / 2); }
// offset of level n in the per-element coefficient list (levels M, M/2, ..., 2)
__host__ __device__ constexpr int s_off(int M, int D, int n) { return n >= M ? 0 : ipow(M / (2 * n), D) + s_off(M, D, 2 * n); }

template <int DIM, int M>
struct Geo {
  static constexpr int MD = ipow(M, DIM);
  static constexpr int NV = DIM + 2;
  static constexpr int P = ipow(M, DIM - 1);
  static constexpr int NL = ilog2(M) + 1;
  static constexpr int NT = MD < 32 ? 32 : MD;
  static constexpr int S = s_total(M, DIM, M);
};

__device__ __forceinline__ const DevLevel& lev(int family, int l) { return c_ops[family].lv[l - 1]; }
__device__ __forceinline__ const DevLevelF& levf(int family, int l) { return c_opsf[family][l - 1]; }

// Index check of the bounds-checked build (-DSESC_BOUNDS, libsesc_bounds.so): an index
// outside [0, n) records flag 8 of the status word (SESC_EBOUNDS) and is replaced by 0,
// so the access stays inside its buffer. The regular build compiles the check out.
__device__ __forceinline__ long long chk(long long i, long long n, long long* status) {
#ifdef SESC_BOUNDS
  if (i < 0 || i >= n) {
    atomicOr((unsigned long long*)status, 8ull);
    return 0;
  }
#endif
  return i;
}

// ---------------------------------------------------------------------------
// element staging: one bulk copy (cp.async.bulk, the TMA engine's untiled mode) of an
// element's contiguous state block from global into this CTA's shared memory,
// completed on an mbarrier. The wait is bounded (KParams::stage_cap polls); a CTA that
// gives up sets flag 4 of the status word (SESC_ETIMEOUT) and skips the element.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* ptr) { return (unsigned)__cvta_generic_to_shared(ptr); }

// Thread 0 arms the barrier and issues the copy (bytes: a multiple of 16; src and dst
// 16-byte aligned); every thread must call stage_wait afterwards. Precondition: a
// __syncthreads since the last generic access to dst. Ends with a block barrier (the
// init is visible before anyone polls).
__device__ __forceinline__ void stage_issue(unsigned long long* bar, void* dst, const void* src, unsigned bytes) {
  if (threadIdx.x == 0) {
    const unsigned b = smem_u32(bar);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
    // order the generic-proxy accesses and the init before the async-proxy copy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(b)
                 : "memory");
  }
  __syncthreads();
}

__device__ __forceinline__ bool stage_poll(unsigned long long* bar) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar))
      : "memory");
  return done != 0;
}

// Waits for the copy (phase 0 of the barrier), at most `cap` polls; returns false,
// block-uniformly, when the wait gave up (the copy then has a second wait of at most
// kStageWaitCap polls to land). The barrier is invalidated before returning, so the
// next element can arm it again.
__device__ __forceinline__ bool stage_wait(unsigned long long* bar, long long* status, long long cap) {
  bool ok = false;
  for (long long it = 0; it < cap; ++it)
    if (stage_poll(bar)) {
      ok = true;
      break;
    }
  if (!ok) {
    for (long long it = 0; it < kStageWaitCap; ++it)
      if (stage_poll(bar)) break;
    if (threadIdx.x == 0) atomicOr((unsigned long long*)status, 4ull);
  }
  const bool all = __syncthreads_and(ok) != 0;
  if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
  return all;
}

// the copy needs 16-byte aligned addresses and a size in 16-byte units
__device__ __forceinline__ bool stage_ok(const void* src, const void* dst, size_t bytes) {
  return ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst) | bytes) & 15) == 0;
}

template <int M>
__device__ __forceinline__ int stride_of(int a) { return a == 0 ? 1 : (a == 1 ? M : M * M); }
template <int M>
__device__ __forceinline__ int coord_of(int t, int a) {
  return a == 0 ? (t % M) : (a == 1 ? (t / M) % M : t / (M * M));
}
// element at coordinate ea along a in the transverse element row tr (the other
// element coordinates in ascending axis order, the lower one fastest), as the face
// kernels number rows
template <int DIM>
__device__ __forceinline__ long long element_of(const KParams& p, int a, int ea, int tr) {
  if (a == 0) return ea + (long long)p.nel[0] * tr;
  if (DIM == 2) return tr + (long long)p.nel[0] * ea;
  if (a == 2) return tr + (long long)p.nel[0] * p.nel[1] * ea;
  return tr % p.nel[0] + (long long)p.nel[0] * (ea + (long long)p.nel[1] * (tr / p.nel[0]));
}

// subcell at coordinate ca along a and transverse point j (the other coordinates in
// ascending axis order, the lower one fastest)
template <int DIM, int M>
__device__ __forceinline__ int subcell_of(int a, int ca, int j) {
  if (DIM == 2) return a == 0 ? ca + M * j : j + M * ca;
  const int j0 = j % M, j1 = j / M;
  return a == 0 ? ca + M * (j0 + M * j1) : (a == 1 ? j0 + M * (ca + M * j1) : j0 + M * (j1 + M * ca));
}

// ---------------------------------------------------------------------------
// Euler physics (eqs. comp-euler-conservative, equation-of-state) and the HLL
// flux with Einfeldt speeds: Roe averages, S_L = min(v_L - c_L, v^ - c^),
// S_R = max(v_R + c_R, v^ + c^); sound speeds sqrt(max(gamma p / rho, 0)) so
// that a squeezed state whose pressure (target 1e-20) rounds below zero gives 0.
// ---------------------------------------------------------------------------
// Entry a of a short register array without a dynamic index (a dynamic index would
// put the array in local memory): the directions are run-time values in the rolled
// direction loops.
template <typename S, int N>
__device__ __forceinline__ S pick(const S (&x)[N], int a) {
  S r = x[0];
#pragma unroll
  for (int k = 1; k < N; ++k)
    if (a == k) r = x[k];
  return r;
}

// Templated on the scalar type S (real here; a dual number in the adjoint).
template <typename S, int DIM>
struct PrimT {
  S rho, inv, v[DIM], p;
  __device__ __forceinline__ void load(const S* q, S g) {
    rho = q[0];
    inv = S(1) / rho;
    S kin = S(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      v[k] = q[1 + k] * inv;
      kin = fma(q[1 + k], v[k], kin);
    }
    p = (g - S(1)) * (q[DIM + 1] - S(0.5) * kin);
  }
};

template <typename S, int DIM>
__device__ __forceinline__ void flux_of_t(const S* q, const PrimT<S, DIM>& w, int a, S* f) {
  const S va = pick(w.v, a);
  S qa = q[1];
#pragma unroll
  for (int k = 1; k < DIM; ++k)
    if (a == k) qa = q[1 + k];
  f[0] = qa;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    f[1 + k] = q[1 + k] * va;
    if (a == k) f[1 + k] = f[1 + k] + w.p;
  }
  f[DIM + 1] = va * (q[DIM + 1] + w.p);
}

template <typename S, int DIM>
__device__ void hll_t(const S* uL, const S* uR, int a, S g, S* F) {
  constexpr int NV = DIM + 2;
  PrimT<S, DIM> L, R;
  L.load(uL, g);
  R.load(uR, g);
  const S cL = sqrt(fmax(g * L.p * L.inv, S(0))), cR = sqrt(fmax(g * R.p * R.inv, S(0)));
  const S HL = (uL[NV - 1] + L.p) * L.inv, HR = (uR[NV - 1] + R.p) * R.inv;
  const S sL = sqrt(L.rho), sR = sqrt(R.rho);
  const S is = S(1) / (sL + sR);
  S vh[DIM], v2 = S(0);
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    vh[k] = (sL * L.v[k] + sR * R.v[k]) * is;
    v2 = fma(vh[k], vh[k], v2);
  }
  const S Hh = (sL * HL + sR * HR) * is;
  const S c2 = (g - S(1)) * (Hh - S(0.5) * v2);
  const S ch = sqrt(fmax(c2, S(0)));
  const S vha = pick(vh, a);
  const S SL = fmin(pick(L.v, a) - cL, vha - ch);
  const S SR = fmax(pick(R.v, a) + cR, vha + ch);
  if (SL >= S(0)) {
    flux_of_t<S, DIM>(uL, L, a, F);
    return;
  }
  if (SR <= S(0)) {
    flux_of_t<S, DIM>(uR, R, a, F);
    return;
  }
  S fL[NV], fR[NV];
  flux_of_t<S, DIM>(uL, L, a, fL);
  flux_of_t<S, DIM>(uR, R, a, fR);
  const S inv = S(1) / (SR - SL);
  const S sls = SL * SR;
#pragma unroll
  for (int v = 0; v < NV; ++v) F[v] = (SR * fL[v] - SL * fR[v] + sls * (uR[v] - uL[v])) * inv;
}

template <int DIM>
using Prim = PrimT<real, DIM>;

template <int DIM>
__device__ __forceinline__ void flux_of(const real* q, const Prim<DIM>& w, int a, real* f) {
  flux_of_t<real, DIM>(q, w, a, f);
}

template <int DIM>
__device__ __forceinline__ void hll(const real* uL, const real* uR, int a, real g, real* F) {
  hll_t<real, DIM>(uL, uR, a, g, F);
}

// FP64 island: permissible set of Sec. 3.1 without a division (rho > 0 and
// 2 rho E > |m|^2). With real = float a test with a relative margin of 1e-4 (far
// above FP32 rounding of these three operations) settles every state outside a
// thin band, and only the band is decided in FP64: the result is the FP64 decision.
template <int DIM>
__device__ __forceinline__ bool permissible64(const real* q) {
  if (sizeof(real) == 4) {
    real m2 = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) m2 = fma(q[1 + k], q[1 + k], m2);
    const real lhs = real(2) * q[0] * q[DIM + 1];
    if (!(q[0] > real(0))) return false;
    if (lhs > m2 * real(1.0001)) return true;
    if (lhs < m2 * real(0.9999)) return false;
  }
  const double r = (double)q[0];
  double m2 = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) m2 = fma((double)q[1 + k], (double)q[1 + k], m2);
  return r > 0.0 && 2.0 * r * (double)q[DIM + 1] > m2;
}

// FP64 island: pressure of a state given in `real`
template <int DIM>
__device__ __forceinline__ double pressure64(const real* q, double g) {
  double kin = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) kin = fma((double)q[1 + k], (double)q[1 + k], kin);
  return (g - 1.0) * ((double)q[DIM + 1] - 0.5 * kin / (double)q[0]);
}

template <int DIM>
__device__ __forceinline__ real pressure_r(const real* q, real g) {
  real kin = 0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) kin = fma(q[1 + k], q[1 + k], kin);
  return (g - real(1)) * (q[DIM + 1] - real(0.5) * kin / q[0]);
}

// pressure at a density-squeezed point (Sec. 2.4 two-step squeezing): the density
// step leaves the lowest point at eps = 1e-20 only up to rounding, and a point
// whose density came out <= 0 is outside the permissible set; its pressure counts
// as -inf (the formula would give a large positive value for rho < 0)
template <int DIM>
__device__ __forceinline__ real squeezed_pressure(const real* q, real g) {
  return q[0] > real(0) ? pressure_r<DIM>(q, g) : real(-INFINITY);
}

// ---------------------------------------------------------------------------
// sub-element bookkeeping
// ---------------------------------------------------------------------------
template <int DIM, int M>
__device__ __forceinline__ int sub_index(int t, int n) {
  const int k = M / n;
  int s = (t % M) / n + k * (((t / M) % M) / n);
  if (DIM == 3) s += k * k * ((t / (M * M)) / n);
  return s;
}
template <int DIM, int M>
__device__ __forceinline__ int local_index(int t, int n) {
  int l = (t % M) % n + n * (((t / M) % M) % n);
  if (DIM == 3) l += n * n * ((t / (M * M)) % n);
  return l;
}
// position of subcell t in the sub-element-contiguous order used by reductions
template <int DIM, int M>
__device__ __forceinline__ int seg_pos(int t, int n) {
  return sub_index<DIM, M>(t, n) * ipow(n, DIM) + local_index<DIM, M>(t, n);
}

// segmented tree reduction over contiguous segments of SZ entries in NVV rows of
// length MD; result at position s*SZ of each row. Includes the barriers.
// Per-sub-element reduction of NVV values per subcell, returned to thread t < NS NVV
// (sub-element t % NS, value t / NS): the warp butterfly below in the FP32 build, a
// packed shared-memory reduction in the FP64 build (every FP64 add there issues for a
// whole warp, so the values are laid out segment by segment and each pass has a thread
// combine 4 consecutive ones: a sub-element of 64 subcells and 4 values takes 12 warp
// instructions of FP64 adds where a halving tree takes 24).
template <int DIM, int M, int N, int NVV, bool MIN, typename T>
__device__ __forceinline__ T tile_reduce(T* x, T* part, int t);

template <int DIM, int M, int N, int NVV, bool MIN>
__device__ __forceinline__ real sub_reduce(real* x, real* red, int t) {
  constexpr int MD = ipow(M, DIM), NS = ipow(M / N, DIM), SZ = ipow(N, DIM), NT = Geo<DIM, M>::NT;
  if (sizeof(real) == 4) return tile_reduce<DIM, M, N, NVV, MIN>(x, red, t);
  if (t < MD) {
    const int pos = seg_pos<DIM, M>(t, N);
#pragma unroll
    for (int v = 0; v < NVV; ++v) red[v * MD + pos] = x[v];
  }
  // red[v MD + s SZ + i]: segment v NS + s holds its SZ values side by side; each pass
  // replaces groups of g consecutive values (inside one segment) by their combination
  constexpr int KMAX = (NVV * MD / 4 + NT - 1) / NT;   // groups per thread in the first pass
  int len = SZ, count = NVV * MD;
#pragma unroll
  for (int pass = 0; pass < 10; ++pass) {
    if (len <= 1) break;
    const int g = len >= 4 ? 4 : 2;
    const int ng = count / g;
    real r[KMAX];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      const int q = t + k * NT;
      if (q < ng) {
        real acc = red[q * g];
        for (int i = 1; i < g; ++i) acc = MIN ? fmin(acc, red[q * g + i]) : acc + red[q * g + i];
        r[k] = acc;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < KMAX; ++k) {
      const int q = t + k * NT;
      if (q < ng) red[q] = r[k];
    }
    len /= g;
    count = ng;
  }
  __syncthreads();
  return (t < NS * NVV) ? red[t] : real(0);
}

// Sum (MIN = false) or minimum over the level-N sub-elements of NVV values per
// subcell; thread t < MD holds x[v] of subcell t (other threads' values are ignored).
// A butterfly over the subcell-index bits that vary inside a sub-element and lie in
// one warp, then the per-warp partials of sub-elements spanning several warps are
// combined through part (at least NVV * MD entries). Thread t < NS * NVV returns the
// result for sub-element t % NS and value t / NS. One barrier; the caller
// synchronises again before part is reused.
template <int DIM, int M, int N, int NVV, bool MIN, typename T>
__device__ __forceinline__ T tile_reduce(T* x, T* part, int t) {
  constexpr int MD = ipow(M, DIM), NS = ipow(M / N, DIM);
  constexpr int LM = ilog2(M), LN = ilog2(N);
  constexpr int SEG = ((1 << LN) - 1) | (DIM >= 2 ? ((1 << LN) - 1) << LM : 0) |
                      (DIM >= 3 ? ((1 << LN) - 1) << (2 * LM) : 0);
  constexpr int INW = SEG & 31, CROSS = SEG & ~31;
  const T neutral = MIN ? T(INFINITY) : T(0);
  if (t >= MD)
#pragma unroll
    for (int v = 0; v < NVV; ++v) x[v] = neutral;
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    if (!((INW >> b) & 1)) continue;
#pragma unroll
    for (int v = 0; v < NVV; ++v) {
      const T y = __shfl_xor_sync(0xffffffffu, x[v], 1 << b);
      x[v] = MIN ? fmin(x[v], y) : x[v] + y;
    }
  }
  constexpr int NC = 1 << cpopc(CROSS);
  if (t < MD && (t & INW) == 0) {
    const int s = sub_index<DIM, M>(t, N);
    int c = 0, k = 0;
#pragma unroll
    for (int b = 5; b < 3 * LM; ++b)
      if ((CROSS >> b) & 1) {
        c |= ((t >> b) & 1) << k;
        ++k;
      }
#pragma unroll
    for (int v = 0; v < NVV; ++v) part[(v * NS + s) * NC + c] = x[v];
  }
  __syncthreads();
  T r = neutral;
  if (t < NS * NVV) {
    r = part[t * NC];
#pragma unroll
    for (int i = 1; i < NC; ++i) r = MIN ? fmin(r, part[t * NC + i]) : r + part[t * NC + i];
  }
  return r;
}

// blockwise n-mode product along axis a: out[v][t] = sum_j A[i][j] in[v][t + (j - i) stride]
template <int DIM, int M, int N, int NVV, typename T>
__device__ __forceinline__ void mode_sq(T* out, const T* in, const T* A, int a, int t) {
  constexpr int MD = ipow(M, DIM);
  if (t >= MD) return;
  const int st = stride_of<M>(a);
  const int i = coord_of<M>(t, a) % N;
  const int base = t - i * st;
#pragma unroll
  for (int v = 0; v < NVV; ++v) {
    T s = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) s = fma(A[i * N + j], in[v * MD + base + j * st], s);
    out[v * MD + t] = s;
  }
}

// reconstruction of the level-N polynomial of every sub-element: ut = u x_0 R x_1 R (x_2 R)
template <int DIM, int M, int N>
__device__ void reconstruct(real* ut, real* tmp, const real* su, int family, int t) {
  constexpr int NV = DIM + 2;
  const real* R = lev(family, ilog2(N)).R;
  if (DIM == 2) {
    mode_sq<DIM, M, N, NV>(tmp, su, R, 0, t);
    __syncthreads();
    mode_sq<DIM, M, N, NV>(ut, tmp, R, 1, t);
    __syncthreads();
  } else {
    mode_sq<DIM, M, N, NV>(ut, su, R, 0, t);
    __syncthreads();
    mode_sq<DIM, M, N, NV>(tmp, ut, R, 1, t);
    __syncthreads();
    mode_sq<DIM, M, N, NV>(ut, tmp, R, 2, t);
    __syncthreads();
  }
}

// value of the level-N polynomial of subcell t's sub-element at interface `row`
// (0..N) along a, from the N means of that row (I_face R of the opgen tables)
template <int DIM, int M, int N>
__device__ __forceinline__ void interface_value(const real* su, int t, int a, int row, int family, real* U) {
  constexpr int MD = ipow(M, DIM);
  constexpr int NV = DIM + 2;
  const real* IRf = lev(family, ilog2(N)).IRf;
  const int st = stride_of<M>(a);
  const int first = t - (coord_of<M>(t, a) % N) * st;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    real s = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) s = fma(IRf[row * N + j], su[v * MD + first + j * st], s);
    U[v] = s;
  }
}

template <int DIM, int M, int N>
__device__ __forceinline__ real interface_density(const real* su, int t, int a, int row, int family) {
  const real* IRf = lev(family, ilog2(N)).IRf;
  const int st = stride_of<M>(a);
  const int first = t - (coord_of<M>(t, a) % N) * st;
  real s = 0;
#pragma unroll
  for (int j = 0; j < N; ++j) s = fma(IRf[row * N + j], su[first + j * st], s);
  return s;
}

// blended state at the right (side = 1) or left (side = 0) face of subcell t along a:
// theta^(1) u_t + sum_n theta^(n) ((1 - beta) <u> + beta U^(n)) (reading R1).
template <int DIM, int M>
__device__ void blended_face_state(const real* su, const real* thtab, const real* beta_s, const real* avg_s,
                                   int t, int a, int side, int family, real* Ub) {
  constexpr int MD = ipow(M, DIM);
  constexpr int NV = DIM + 2;
  constexpr int NL = ilog2(M) + 1;
  constexpr int S = s_total(M, DIM, M);
  const real th1 = thtab[t];
#pragma unroll
  for (int v = 0; v < NV; ++v) Ub[v] = (th1 != real(0)) ? th1 * su[v * MD + t] : real(0);
  const int c = coord_of<M>(t, a);
#pragma unroll
  for (int l = 1; l < NL; ++l) {
    const real th = thtab[l * MD + t];
    if (th == real(0)) continue;
    const int n = 1 << l;
    const int row = (c % n) + side;
    real U[NV];
    if (n == 2) interface_value<DIM, M, 2>(su, t, a, row, family, U);
    else if (n == 4) interface_value<DIM, M, 4>(su, t, a, row, family, U);
    else interface_value<DIM, M, (M >= 8 ? 8 : 4)>(su, t, a, row, family, U);
    const int s = sub_index<DIM, M>(t, n);
    const int off = s_off(M, DIM, n);
    const real b = beta_s[off + s];
    if (b != real(1)) {
#pragma unroll
      for (int v = 0; v < NV; ++v) U[v] = (real(1) - b) * avg_s[v * S + off + s] + b * U[v];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) Ub[v] += th * U[v];
  }
}

// ---------------------------------------------------------------------------
// Blended common flux on a group of NF faces with P transverse points each
// (readings R2 / R7). Thread tid < NF*P handles face f = tid / P, point j = tid % P.
// Scratch: sUL, sUR, sT, sF each NF*NV*P reals, sflag NF*P ints.
// ---------------------------------------------------------------------------
template <int DIM, int M, int N>
__device__ __forceinline__ void transverse(const real* src, real* sT, const real* A, int f, int j, bool valid,
                                           real* out) {
  constexpr int NV = DIM + 2;
  constexpr int P = ipow(M, DIM - 1);
  if (DIM == 2) {
    if (valid) {
      const int i = j % N, base = j - i;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        real s = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) s = fma(A[i * N + k], src[(f * NV + v) * P + base + k], s);
        out[v] = s;
      }
    }
  } else {
    if (valid) {
      const int i0 = (j % M) % N, b0 = j - i0;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        real s = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) s = fma(A[i0 * N + k], src[(f * NV + v) * P + b0 + k], s);
        sT[(f * NV + v) * P + j] = s;
      }
    }
    __syncthreads();
    if (valid) {
      const int i1 = (j / M) % N, b1 = j - i1 * M;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        real s = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) s = fma(A[i1 * N + k], sT[(f * NV + v) * P + b1 + k * M], s);
        out[v] = s;
      }
    }
    __syncthreads();
  }
}

template <int DIM, int M, int N>
__device__ void level_candidate(const real* UL, const real* UR, real wl, int a, real g, int family, int f, int j,
                                bool valid, real* sUL, real* sUR, real* sT, real* sF, int* sflag, bool& have1,
                                real* F1, real* Fout, long long* counters) {
  constexpr int NV = DIM + 2;
  constexpr int P = ipow(M, DIM - 1);
  const DevLevel& L = lev(family, ilog2(N));
  real rL[NV], rR[NV];
  transverse<DIM, M, N>(sUL, sT, L.R, f, j, valid, rL);
  transverse<DIM, M, N>(sUR, sT, L.R, f, j, valid, rR);
  const bool ok = valid && permissible64<DIM>(rL) && permissible64<DIM>(rR);
  if (valid) sflag[f * P + j] = ok ? 1 : 0;
  __syncthreads();
  bool blk = valid;
  if (valid) {
    if (DIM == 2) {
      const int b = j - j % N;
      for (int k = 0; k < N; ++k) blk = blk && sflag[f * P + b + k];
    } else {
      const int b = j - (j % M) % N - ((j / M) % N) * M;
      for (int k1 = 0; k1 < N; ++k1)
        for (int k0 = 0; k0 < N; ++k0) blk = blk && sflag[f * P + b + k0 + k1 * M];
    }
  }
  real Fn[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Fn[v] = 0;
  if (blk) hll<DIM>(rL, rR, a, g, Fn);
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) sF[(f * NV + v) * P + j] = Fn[v];
  }
  __syncthreads();
  real Fp[NV];
  transverse<DIM, M, N>(sF, sT, L.P, f, j, valid, Fp);
  if (valid && wl != real(0)) {
    if (blk) {
#pragma unroll
      for (int v = 0; v < NV; ++v) Fout[v] += wl * Fp[v];
    } else {
      if (!have1) {
        hll<DIM>(UL, UR, a, g, F1);
        have1 = true;
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) Fout[v] += wl * F1[v];
      // one count per transverse block: its first point
      const bool first = (DIM == 2) ? (j % N == 0) : ((j % M) % N == 0 && ((j / M) % N) == 0);
      if (first) atomicAdd((unsigned long long*)&counters[2], 1ull);
    }
  }
  __syncthreads();
}

template <int DIM, int M>
__device__ void blended_flux(const real* UL, const real* UR, const real* w, int a, real g, int family, int f, int j,
                             bool valid, real* sUL, real* sUR, real* sT, real* sF, int* sflag, real* Fout,
                             long long* counters) {
  constexpr int NV = DIM + 2;
  constexpr int P = ipow(M, DIM - 1);
  constexpr int NL = ilog2(M) + 1;
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      sUL[(f * NV + v) * P + j] = UL[v];
      sUR[(f * NV + v) * P + j] = UR[v];
    }
  }
  real F1[NV];
  bool have1 = false;
#pragma unroll
  for (int v = 0; v < NV; ++v) Fout[v] = 0;
  if (valid && w[0] != real(0)) {
    hll<DIM>(UL, UR, a, g, F1);
    have1 = true;
#pragma unroll
    for (int v = 0; v < NV; ++v) Fout[v] = w[0] * F1[v];
  }
  __syncthreads();
#pragma unroll
  for (int l = 1; l < NL; ++l) {
    if (!__syncthreads_or(valid && w[l] != real(0))) continue;
    if (l == 1)
      level_candidate<DIM, M, 2>(UL, UR, w[l], a, g, family, f, j, valid, sUL, sUR, sT, sF, sflag, have1, F1, Fout,
                                 counters);
    else if (l == 2)
      level_candidate<DIM, M, 4>(UL, UR, w[l], a, g, family, f, j, valid, sUL, sUR, sT, sF, sflag, have1, F1, Fout,
                                 counters);
    else
      level_candidate<DIM, M, (M >= 8 ? 8 : 4)>(UL, UR, w[l], a, g, family, f, j, valid, sUL, sUR, sT, sF, sflag,
                                                have1, F1, Fout, counters);
  }
}

// blending weights per subcell from the snapped alpha (eq. blending-weights)
template <int DIM, int M>
__device__ __forceinline__ void weights_of(const double* alpha, int t, double* thl) {
  constexpr int NL = ilog2(M) + 1;
  double rest = 1.0;
#pragma unroll
  for (int l = NL - 1; l >= 1; --l) {
    const int n = 1 << l;
    const double A = alpha[s_off(M, DIM, n) + sub_index<DIM, M>(t, n)];
    // a snapped factor (0 or 1, recognised from its bits on the integer units) needs no
    // FP64 arithmetic: A rest and rest (1 - A) are then exact
    const long long bits = __double_as_longlong(A);
    if (bits == 0ll) {
      thl[l] = 0.0;
    } else if (bits == 0x3FF0000000000000ll) {
      thl[l] = rest;
      rest = 0.0;
    } else {
      thl[l] = A * rest;
      rest = rest * (1.0 - A);
    }
  }
  thl[0] = rest;
}

// ---------------------------------------------------------------------------
// K1: indicator, coefficients, blending weights and element face states
// ---------------------------------------------------------------------------
template <int DIM, int M>
struct K1Smem {
  static constexpr int MD = Geo<DIM, M>::MD, NV = Geo<DIM, M>::NV, S = Geo<DIM, M>::S, NL = Geo<DIM, M>::NL;
  // doubles first, then reals
  static constexpr int d_alpha = 0;
  static constexpr int d_beta = d_alpha + S;
  static constexpr int d_brho = d_beta + S;
  static constexpr int d_eps = d_brho + S;       // eps per sub-element of the current level
  static constexpr int d_red = d_eps + S;        // MD doubles (blending-factor staging)
  static constexpr int d_total = d_red + MD;
  static constexpr int r_su = 0;
  static constexpr int r_ut = r_su + NV * MD;
  static constexpr int r_tmp = r_ut + NV * MD;
  static constexpr int r_red = r_tmp + NV * MD;
  static constexpr int r_th = r_red + NV * MD;
  static constexpr int r_avg = r_th + NL * MD;
  static constexpr int r_sig = r_avg + NV * S;
  static constexpr int r_alf = r_sig + NV * S;                // alpha, beta in the compute type
  static constexpr int r_bef = r_alf + S;
  static constexpr int r_bnd = r_bef + S;                    // element bounds for the squeeze test
  static constexpr int r_total = r_bnd + 2 * NV * (Geo<DIM, M>::NT / 32);
  static constexpr size_t bytes = sizeof(double) * d_total + sizeof(real) * r_total;
};

// per-sub-element averages of level N into avg[v][off + s]
template <int DIM, int M, int N>
__device__ void sub_averages(const real* su, real* red, real* avg, int t) {
  constexpr int MD = ipow(M, DIM), NV = DIM + 2, S = Geo<DIM, M>::S;
  constexpr int SZ = ipow(N, DIM);
  constexpr int NS = ipow(M / N, DIM);
  constexpr int off = s_off(M, DIM, N);
  __syncthreads();
  real x[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) x[v] = (t < MD) ? su[v * MD + t] : real(0);
  const real r = sub_reduce<DIM, M, N, NV, false>(x, red, t);
  if (t < NS * NV) {
    const int v = t / NS, s = t % NS;
    avg[v * S + off + s] = r / real(SZ);
  }
  __syncthreads();
}

// sigma^(N) per primitive variable and sub-element (reading R3), from ut (unlimited nodal)
template <int DIM, int M, int N>
__device__ void smoothness(const real* ut, real* tmp, real* red, real* sig, real g, int family, int t) {
  constexpr int MD = ipow(M, DIM), NV = DIM + 2, S = Geo<DIM, M>::S;
  constexpr int SZ = ipow(N, DIM);
  constexpr int NS = ipow(M / N, DIM);
  constexpr int off = s_off(M, DIM, N);
  const DevLevel& L = lev(family, ilog2(N));
  if (t < MD) {
    real q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = ut[v * MD + t];
    Prim<DIM> w;
    w.load(q, g);
    tmp[t] = q[0];
#pragma unroll
    for (int k = 0; k < DIM; ++k) tmp[(1 + k) * MD + t] = w.v[k];
    tmp[(NV - 1) * MD + t] = w.p;
  }
  __syncthreads();
  real acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0;
  if (t < MD) {
    real W = L.w[(t % M) % N] * L.w[((t / M) % M) % N];
    if (DIM == 3) W *= L.w[(t / (M * M)) % N];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int st = stride_of<M>(a);
      const int i = coord_of<M>(t, a) % N, base = t - i * st;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        real s = 0;
#pragma unroll
        for (int j = 0; j < N; ++j) s = fma(L.Dn[i * N + j], tmp[v * MD + base + j * st], s);
        acc[v] += fabs(s) * W;
      }
    }
  }
  const real r = sub_reduce<DIM, M, N, NV, false>(acc, red, t);
  if (t < NS * NV) {
    const int v = t / NS, s = t % NS;
    const real h = real(N) / real(M);
    const real hd = (DIM == 2) ? h : h * h;
    sig[v * S + off + s] = hd * r;
  }
  __syncthreads();
}

// eps = min(1e-20, <rho>, <p>) of eq. calc-squeezing-parameter (FP64 result). With
// real = float a test with a wide margin settles the common case eps = 1e-20 in
// FP32; otherwise <p> >= 1e-20 is tested without a division, (gamma-1)(2 rho E -
// |m|^2) >= 2 rho 1e-20, and the pressure is divided out only when it is that small.
template <int DIM>
__device__ __forceinline__ double eps_of_average(const real* q, double g) {
  if (sizeof(real) == 4) {
    real m2 = 0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) m2 = fma(q[1 + k], q[1 + k], m2);
    const real e2 = real(2) * q[0] * q[DIM + 1] - m2;
    if (q[0] > real(1e-18) && real(g - 1.0) * e2 > real(1.01) * real(2e-18) * q[0] && e2 > real(1e-6) * m2)
      return 1e-20;
  }
  const double r = (double)q[0];
  double m2 = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) m2 = fma((double)q[1 + k], (double)q[1 + k], m2);
  const double e2 = 2.0 * r * (double)q[DIM + 1] - m2;
  if (r >= 1e-20 && (g - 1.0) * e2 >= 2e-20 * r) return 1e-20;
  return fmin(fmin(1e-20, r), pressure64<DIM>(q, g));
}

// squeezing parameter beta^(N) per sub-element (reading R4, two steps): point
// values and minima in the compute type, the formula in FP64; the ratios are only
// divided out when a minimum falls below eps
template <int DIM, int M, int N>
__device__ void squeeze(const real* su, const real* ut, real* red, const real* avg, double* beta, double* brho,
                        double* epsv, double g, int family, int t, long long* counters) {
  constexpr int MD = ipow(M, DIM), NV = DIM + 2, S = Geo<DIM, M>::S;
  constexpr int SZ = ipow(N, DIM);
  constexpr int NS = ipow(M / N, DIM);
  constexpr int off = s_off(M, DIM, N);
  const int s = (t < MD) ? sub_index<DIM, M>(t, N) : 0;
  const int pos = (t < MD) ? seg_pos<DIM, M>(t, N) : 0;
  // step 1: density minimum over nodes and owned face points
  real xr[1] = {real(INFINITY)};
  if (t < MD) {
    real rmin = ut[t];
#pragma unroll 1
    for (int a = 0; a < DIM; ++a) {
      const int i = coord_of<M>(t, a) % N;
      rmin = fmin(rmin, interface_density<DIM, M, N>(su, t, a, i, family));
      if (i == N - 1) rmin = fmin(rmin, interface_density<DIM, M, N>(su, t, a, N, family));
    }
    xr[0] = rmin;
  }
  const real rmin_s = sub_reduce<DIM, M, N, 1, true>(xr, red, t);
  if (t < NS) {
    real q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = avg[v * S + off + t];
    const double eps = eps_of_average<DIM>(q, g);
    epsv[t] = eps;
    const real rminr = rmin_s;
    double b = 1.0;
    // rmin >= eps settles in the compute type unless rmin lies within a factor 2 of 1e-20
    if (!(rminr >= real(2e-20)) || eps != 1e-20) {
      const double rmin = (double)rminr;
      if (!(rmin >= eps)) b = fmin(((double)q[0] - eps) / ((double)q[0] - rmin), 1.0);
    }
    brho[off + t] = b;
  }
  __syncthreads();
  // step 2: pressure minimum over the density-squeezed points
  if (t < MD) {
    const real br = (real)brho[off + s];
    real av[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) av[v] = avg[v * S + off + s];
    real q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = (br == real(1)) ? ut[v * MD + t] : (real(1) - br) * av[v] + br * ut[v * MD + t];
    real pmin = squeezed_pressure<DIM>(q, (real)g);
#pragma unroll 1
    for (int a = 0; a < DIM; ++a) {
      const int i = coord_of<M>(t, a) % N;
      for (int side = 0; side < 2; ++side) {
        if (side == 1 && i != N - 1) break;
        real U[NV];
        interface_value<DIM, M, N>(su, t, a, i + side, family, U);
        if (br != real(1)) {
#pragma unroll
          for (int v = 0; v < NV; ++v) U[v] = (real(1) - br) * av[v] + br * U[v];
        }
        pmin = fmin(pmin, squeezed_pressure<DIM>(U, (real)g));
      }
    }
    xr[0] = pmin;
  }
  const real pmin_s = sub_reduce<DIM, M, N, 1, true>(xr, red, t);
  if (t < NS) {
    real q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = avg[v * S + off + t];
    const double eps = epsv[t];
    const real pminr = pmin_s;
    double bp = 1.0;
    if (!(pminr >= real(2e-20)) || eps != 1e-20) {
      const double pmin = (double)pminr;
      if (!(pmin >= eps)) {
        const double pavg = pressure64<DIM>(q, g);
        bp = fmin((pavg - eps) / (pavg - pmin), 1.0);
      }
    }
    double b = brho[off + t];
    if (bp != 1.0) b *= bp;
    if (b != 1.0) {
      if (!permissible64<DIM>(q) || !isfinite(b)) b = 0.0;
      b = fmax(b, 0.0);
    } else if (!permissible64<DIM>(q)) {
      b = 0.0;
    }
    beta[off + t] = b;
    if (b < 1.0) atomicAdd((unsigned long long*)&counters[1], 1ull);
  }
  __syncthreads();
}

// raw blending factor of level NP (= 2 N) from sigma^(NP), the children sums of
// sigma^(N) and beta^(NP) (eq. calc-blending-factor). One lane per (sub-element,
// primitive variable) computes the ratio in FP64; the minimum over the variables
// goes through `stage` (NV * (M/NP)^DIM doubles).
// threshold-near test of the decisions (counted per element): a raw factor within 1e-10
// of alpha_H or alpha_L, or a squeezing parameter within 1e-10 of beta_L
__device__ __forceinline__ bool near_threshold(double a, double b, const KParams& p) {
  return fabs(a - p.alphaH) < 1e-10 || fabs(a - p.alphaL) < 1e-10 || fabs(b - p.betaL) < 1e-10;
}

template <int DIM, int M, int NP>
__device__ void blending_factor(const real* sig, const double* beta, double* alpha, double* stage, double tauA,
                                double tauS, double betaL, int t, const KParams& par, bool& near) {
  constexpr int NV = DIM + 2, S = Geo<DIM, M>::S;
  constexpr int NSP = ipow(M / NP, DIM);
  constexpr int kp = M / NP, kc = M / (NP / 2);
  constexpr int offp = s_off(M, DIM, NP), offc = s_off(M, DIM, NP / 2);
  if (t < NSP * NV) {
    const int sp_i = t / NV, v = t % NV;
    const int px = sp_i % kp, py = (sp_i / kp) % kp, pz = (DIM == 3) ? sp_i / (kp * kp) : 0;
    // children sum: pairs along x, then y, then z
    real yz[2][2];
    for (int dz = 0; dz < (DIM == 3 ? 2 : 1); ++dz)
      for (int dy = 0; dy < 2; ++dy) {
        const int cx = 2 * px, cy = 2 * py + dy, cz = 2 * pz + dz;
        const int c0 = cx + kc * (cy + kc * cz);
        yz[dz][dy] = sig[v * S + offc + c0] + sig[v * S + offc + c0 + 1];
      }
    real csr = yz[0][0] + yz[0][1];
    if (DIM == 3) csr = csr + (yz[1][0] + yz[1][1]);
    const real spr = sig[v * S + offp + sp_i];
    double av = 0.0;
    if (isfinite(spr) && isfinite(csr)) {
      bool done = false;
      if (sizeof(real) == 4) {
        // outside the transition band tau_S < ratio < tau_S + 1/tau_A the factor is
        // exactly 1 or 0; the FP32 ratio is within 1e-6 of the exact one, so it
        // settles those cases and the FP64 ratio is formed only inside the band
        const real r32 = fabs(spr - csr) / fmax(fmax(spr, csr), real(1));
        if (r32 < real(tauS) * real(0.999999)) {
          av = 1.0;
          done = true;
        } else if (r32 > real(tauS + 1.0 / tauA) * real(1.000001)) {
          done = true;
        }
      }
      if (!done) {
        const double den = (double)fmax(fmax(spr, csr), real(1));
        const double ratio = fabs((double)spr - (double)csr) / den;
        if (isfinite(ratio)) av = 1.0 - fmin(fmax(tauA * (ratio - tauS), 0.0), 1.0);
      }
    }
    stage[t] = av;
  }
  __syncthreads();
  if (t < NSP) {
    double amin = stage[t * NV];
#pragma unroll
    for (int v = 1; v < NV; ++v) amin = fmin(amin, stage[t * NV + v]);
    if (beta[offp + t] < betaL) amin = 0.0;
    alpha[offp + t] = amin;
    near = near || near_threshold(amin, beta[offp + t], par);
  }
  __syncthreads();
}

// snap level n; returns true if all sub-elements exceeded alpha_H (the loop ends)
template <int DIM, int M, int N>
__device__ bool snap(double* alpha, double alphaH, double alphaL, int t) {
  constexpr int NS = ipow(M / N, DIM);
  constexpr int off = s_off(M, DIM, N);
  bool hi = true, lo = true;
  if (t < NS) {
    const double a = alpha[off + t];
    hi = a > alphaH;
    lo = a < alphaL;
  }
  const bool all_hi = __syncthreads_and(hi);
  const bool all_lo = __syncthreads_and(lo);
  if (t < NS) {
    if (all_hi) alpha[off + t] = 1.0;
    else if (all_lo) alpha[off + t] = 0.0;
  }
  __syncthreads();
  return all_hi;
}

template <int DIM, int M, int N>
__device__ void level_stats(const real* su, real* ut, real* tmp, real* red, real* avg, real* sig, real g, int family,
                            int t) {
  sub_averages<DIM, M, N>(su, red, avg, t);
  reconstruct<DIM, M, N>(ut, tmp, su, family, t);
  smoothness<DIM, M, N>(ut, tmp, red, sig, g, family, t);
}

// Levels whose squeezing would certainly leave beta = 1 (Sec. 2.4): every point the
// squeezing checks at level n (nodal values, subcell-face values) is a combination
// of the element's means with weights that sum to 1 and whose absolute values sum
// to at most Lambda_n = max(lamR^d, lamI), so each of its variables lies within
// Lambda_n times the half-range of that variable around its mid-range. When the
// density and the pressure of every state in that box exceed the largest possible
// eps (1e-20), with margins for the rounding of the point values, every ratio of
// eq. calc-squeezing-parameter is 1 and the level is skipped. Returns a CTA-uniform
// bit mask over levels (bit l for n = 2^l); bnd holds 2 NV (NT/32) reals.
// order-preserving integer key of a double (non-NaN): min / max of the keys as signed
// integers are the min / max of the values, formed on the integer units
__device__ __forceinline__ long long dkey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7FFFFFFFFFFFFFFFll);
}
__device__ __forceinline__ double dunkey(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFll));
}

template <int DIM, int M>
__device__ int squeeze_free_levels(const real* su, real* bnd, real g, int family, int t) {
  constexpr int MD = Geo<DIM, M>::MD, NV = Geo<DIM, M>::NV, NT = Geo<DIM, M>::NT, NL = Geo<DIM, M>::NL;
  constexpr int NW = NT / 32;
  real lo[NV], hi[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const real x = su[v * MD + (t < MD ? t : 0)];
    const bool fin = isfinite(x);   // a non-finite mean makes the range infinite: no skip
    lo[v] = fin ? x : real(-INFINITY);
    hi[v] = fin ? x : real(INFINITY);
  }
  if (sizeof(real) == 8) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      long long kl = dkey((double)lo[v]), kh = dkey((double)hi[v]);
#pragma unroll
      for (int o = 16; o > 0; o /= 2) {
        kl = min(kl, __shfl_xor_sync(0xffffffffu, kl, o));
        kh = max(kh, __shfl_xor_sync(0xffffffffu, kh, o));
      }
      lo[v] = (real)dunkey(kl);
      hi[v] = (real)dunkey(kh);
    }
  } else {
#pragma unroll
    for (int o = 16; o > 0; o /= 2)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        lo[v] = fmin(lo[v], __shfl_xor_sync(0xffffffffu, lo[v], o));
        hi[v] = fmax(hi[v], __shfl_xor_sync(0xffffffffu, hi[v], o));
      }
  }
  const int lane = t % 32, wid = t / 32;
  if (lane == 0)
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      bnd[(2 * v) * NW + wid] = lo[v];
      bnd[(2 * v + 1) * NW + wid] = hi[v];
    }
  __syncthreads();
  // lane l - 1 of the first warp tests level l; the mask goes to every thread by a vote
  const int l = t + 1;
  bool ok = false;
  if (l < NL) {
#pragma unroll
    for (int v = 0; v < NV; ++v)
      for (int k = 0; k < NW; ++k) {
        lo[v] = fmin(lo[v], bnd[(2 * v) * NW + k]);
        hi[v] = fmax(hi[v], bnd[(2 * v + 1) * NW + k]);
      }
    const real eps_r = sizeof(real) == 4 ? real(6e-8) : real(1.2e-16);
    const DevLevel& L = lev(family, l);
    real lamd = L.lamR;
    for (int k = 1; k < DIM; ++k) lamd *= L.lamR;
    const real Lam = fmax(lamd, L.lamI) * real(1.001);
    real c[NV], B[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      c[v] = real(0.5) * (lo[v] + hi[v]);
      B[v] = Lam * real(0.5) * (hi[v] - lo[v]) + real(64) * eps_r * Lam * fmax(fabs(lo[v]), fabs(hi[v]));
    }
    const real rlo = c[0] - B[0];
    const real Elo = c[NV - 1] - B[NV - 1];
    ok = rlo >= real(4e-20) && Elo > real(0);
    if (ok) {
      real m2 = 0;
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        const real m = fabs(c[1 + k]) + B[1 + k];
        m2 = fma(m, m, m2);
      }
      const real kin = m2 / (real(2) * rlo);
      const real plo = (g - real(1)) * (Elo - kin);
      ok = plo >= real(4e-20) && plo >= real(1e-4) * (g - real(1)) * (fabs(hi[NV - 1]) + kin);
    }
  }
  int mask = 0;
#pragma unroll
  for (int k = 1; k < NL; ++k) mask |= __syncthreads_or(ok && l == k) ? (1 << k) : 0;
  return mask;
}

// ---------------------------------------------------------------------------
// Certified FP32 pass of the FP64 indicator (FP64 build). GB300 issues FP32
// arithmetic at about 64 times its FP64 rate, and the smoothness statistics of
// eq. L1-norm-slope (reconstruction, primitive variables, derivative L1 norms) are
// most of the indicator's FP64 work. Their only use is the raw blending factor of
// eq. calc-blending-factor, which is exactly 1 below the transition band (ratio <=
// tau_S) and exactly 0 above it (ratio >= tau_S + 1/tau_A). This pass forms every
// sigma in FP32 with a bound that covers both its own error and the error of the
// FP64 evaluation against the exact value from the FP64 means, and decides a factor
// only where the whole interval of possible ratios lies outside the band with a
// margin of 1e-6 relative: there the FP64 evaluation yields the same 0 or 1. The
// squeezing of eq. calc-squeezing-parameter is certified the same way to leave
// beta = 1 (level_sigma_f32). An element where a factor that the snapping loop
// visits stays undecided, or a squeezing it reaches is not certified, takes the FP64
// evaluation from the start, so every coefficient is the one of the FP64 path bit
// for bit.
//
// The reconstruction runs on the deviations d = u - r of the means from one
// reference value r per variable (the element's first mean, exact in FP32): the
// operators reproduce constants (R 1 = 1, D 1 = 0), so the nodal values are r plus
// the reconstruction of d and the derivatives are those of w - c for any constant c
// of a row (its first node), and the FP32 errors scale with the variation inside the
// element instead of its magnitude. Bounds, first order in u = 2^-24 with 1 % added
// for the higher orders:
// - nodal values: d (N + 2) u Lam_R^d Q'_v + u |value|, Lam_R = largest absolute
//   row sum of R, Q'_v = max |d_v| over the element + 2^-28 max |u_v| (the second
//   term covers the FP64 evaluation, whose reconstruction carries the same bound
//   with 2^-53 on the magnitudes);
// - primitives: rho as its value (the pass requires e_rho <= 1e-3 rho); v_k =
//   m_k / rho: (e_m + |v_k| e_rho) / rho + 4 u |v_k|; kin = m.v: sum of |m_k| e_vk +
//   |v_k| e_mk + e_mk e_vk + (d + 1) u |m_k v_k|; p = (g - 1)(E - kin/2):
//   (g - 1)(e_E + e_kin / 2) plus (2 u + the relative rounding of g - 1) |p|;
// - derivative at a node: sum_j |D_kj| (e_w,j + (N + 3) u |w_j - c| + (N + 3) 2^-53
//   |w_j|) (the FMA chains of both evaluations and the rounded operator); sigma's
//   bound sums these with the quadrature weights like sigma itself;
// - the sums forming sigma (positive terms, at most d + M^d + 8 roundings) add
//   (d + M^d + 8) u sigma.
// ---------------------------------------------------------------------------
template <int DIM, int M>
struct F32Scratch {   // offsets in floats from the pass's scratch base
  static constexpr int MD = Geo<DIM, M>::MD, NV = Geo<DIM, M>::NV, S = Geo<DIM, M>::S;
  static constexpr int NW = Geo<DIM, M>::NT / 32;
  static constexpr int sf = 0;                  // deviations of the means from ref, FP32
  static constexpr int ut = sf + NV * MD;       // reconstruction, then the per-node value bounds
  static constexpr int tmp = ut + NV * MD;      // primitives
  static constexpr int red = tmp + NV * MD;     // two reduction buffers of NV MD
  static constexpr int sg = red + 2 * NV * MD;  // sigma [v][S]
  static constexpr int eg = sg + NV * S;        // bound of sigma's error [v][S]
  static constexpr int code = eg + NV * S;      // decision per (sub-element, variable), as int
  static constexpr int qw = code + NV * S;      // per-warp maxima of |d| and |u|: [2 NV][NW]
  static constexpr int q = qw + 2 * NV * NW;    // Q'_v
  static constexpr int ref = q + NV;            // reference value per variable
  static constexpr int total = ref + NV;
};

// primitive variables (rho, v, p) of a state q given in FP32 with the bounds e of
// its errors, and bounds b of their errors (the rules above); false where rho <= 0,
// e_rho > 1e-3 rho or a value is not finite. lim: a bound of |E| + kin.
template <int DIM>
__device__ __forceinline__ bool prim_bound_f32(const float* q, const float* e, float g, float* w, float* b,
                                               float& lim) {
  constexpr int NV = DIM + 2;
  constexpr float u = 0x1p-24f;
  const float rho = q[0];
  const float er = e[0];
  bool ok = rho > 0.f && er <= 1e-3f * rho;
  const float inv = 1.0f / rho;
  float vel[DIM], ev[DIM], kin = 0.f, ekin = 0.f, mv = 0.f;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    vel[k] = q[1 + k] * inv;
    kin = fmaf(q[1 + k], vel[k], kin);
  }
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const float em = e[1 + k];
    ev[k] = 1.003f * (em + fabsf(vel[k]) * er) * inv + 4.f * u * fabsf(vel[k]);
    ekin += fabsf(q[1 + k]) * ev[k] + fabsf(vel[k]) * em + em * ev[k];
    mv += fabsf(q[1 + k] * vel[k]);
  }
  ekin = 1.001f * ekin + float(DIM + 1) * u * mv;
  const float gm1 = g - 1.f;
  const float p = gm1 * (q[NV - 1] - 0.5f * kin);
  const float grel = 2.02f * u * g / gm1;   // |fl(g) - 1 - (gamma - 1)| / (gamma - 1)
  const float ep = 1.001f * gm1 * (e[NV - 1] + 0.5f * ekin) + (2.01f * u + grel) * fabsf(p);
  w[0] = rho;
  b[0] = er;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    w[1 + k] = vel[k];
    b[1 + k] = ev[k];
  }
  w[NV - 1] = p;
  b[NV - 1] = ep;
  lim = 1.01f * (fabsf(q[NV - 1]) + e[NV - 1] + kin + ekin);
#pragma unroll
  for (int v = 0; v < NV; ++v) ok = ok && isfinite(w[v]) && isfinite(b[v]);
  return ok && isfinite(lim);
}

// sigma^(N) and its error bound per primitive variable and sub-element into
// sg / eg [v][off + s]. With sq set, also certifies that the squeezing of this level
// leaves beta = 1 (eq. calc-squeezing-parameter): density and pressure at least
// 2e-20 at every node and owned subcell-face value, for the FP64 evaluation too (so
// both of its minima clear eps <= 1e-20), and nodal pressures at least 1e-13 (g - 1)
// (|E| + kin), which keeps the FP64 permissibility test of the sub-element average
// (the Gauss-weighted nodal average: p is concave, kin convex) clear of its rounding.
// Returns (CTA-uniform) 0 where a bound cannot be formed, 2 where the statistics
// are bounded but beta = 1 is not certified, 1 otherwise.
template <int DIM, int M, int N>
__device__ int level_sigma_f32(float* fs, float g, int family, bool sq, int t) {
  using F = F32Scratch<DIM, M>;
  constexpr int MD = F::MD, NV = F::NV, S = F::S;
  constexpr int NS = ipow(M / N, DIM);
  constexpr int off = s_off(M, DIM, N);
  constexpr float u = 0x1p-24f;
  const DevLevelF& L = levf(family, ilog2(N));
  float* sf = fs + F::sf;
  float* ut = fs + F::ut;
  float* tmp = fs + F::tmp;
  float* red = fs + F::red;
  // reconstruction of the deviations, every sub-element's level-N polynomial
  if (DIM == 2) {
    mode_sq<DIM, M, N, NV>(tmp, (const float*)sf, L.R, 0, t);
    __syncthreads();
    mode_sq<DIM, M, N, NV>(ut, (const float*)tmp, L.R, 1, t);
  } else {
    mode_sq<DIM, M, N, NV>(ut, (const float*)sf, L.R, 0, t);
    __syncthreads();
    mode_sq<DIM, M, N, NV>(tmp, (const float*)ut, L.R, 1, t);
    __syncthreads();
    mode_sq<DIM, M, N, NV>(ut, (const float*)tmp, L.R, 2, t);
  }
  __syncthreads();
  bool ok = true, sqok = true;
  if (t < MD) {
    float lamd = L.lamR;
#pragma unroll
    for (int k = 1; k < DIM; ++k) lamd *= L.lamR;
    const float cR = 1.01f * float(DIM * (N + 2)) * u * lamd;
    float q[NV], e[NV], w[NV], b[NV], lim;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      q[v] = fs[F::ref + v] + ut[v * MD + t];
      e[v] = cR * fs[F::q + v] + 1.01f * u * fabsf(q[v]);
    }
    ok = prim_bound_f32<DIM>(q, e, g, w, b, lim);
    if (sq) {
      const float pl = w[NV - 1] - b[NV - 1];
      sqok = w[0] - b[0] >= 2e-20f && pl >= 2e-20f && pl >= 1e-13f * (g - 1.f) * lim;
      // owned subcell-face values along every direction (the left face of each
      // subcell, the right one of a sub-element's last): I_face R of the row's means
      const float cI = 1.01f * float(N + 2) * u * L.lamI;
#pragma unroll 1
      for (int a = 0; a < DIM; ++a) {
        const int st = stride_of<M>(a);
        const int i = coord_of<M>(t, a) % N, first = t - i * st;
        for (int side = 0; side < 2; ++side) {
          if (side == 1 && i != N - 1) break;
          const int row = i + side;
          float U[NV], eU[NV], wf[NV], bf[NV], lf;
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < N; ++j) s = fmaf(L.IRf[row * N + j], sf[v * MD + first + j * st], s);
            U[v] = fs[F::ref + v] + s;
            eU[v] = cI * fs[F::q + v] + 1.01f * u * fabsf(U[v]);
          }
          const bool okf = prim_bound_f32<DIM>(U, eU, g, wf, bf, lf);
          sqok = sqok && okf && wf[0] - bf[0] >= 2e-20f && wf[NV - 1] - bf[NV - 1] >= 2e-20f;
        }
      }
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      tmp[v * MD + t] = w[v];
      ut[v * MD + t] = b[v];   // this thread's own entries: read above, by no other thread
    }
  }
  if (!__syncthreads_and(ok)) return 0;
  const bool sq_all = __syncthreads_and(sqok);
  // quadrature-weighted L1 norms of the derivatives (sigma) and of their error bounds
  constexpr float cw = float(N + 3) * u, cw64 = float(N + 3) * 0x1p-53f;
  float acc[NV], accb[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = accb[v] = 0.f;
  if (t < MD) {
    float W = L.w[(t % M) % N] * L.w[((t / M) % M) % N];
    if (DIM == 3) W *= L.w[(t / (M * M)) % N];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int st = stride_of<M>(a);
      const int i = coord_of<M>(t, a) % N, base = t - i * st;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const float c = tmp[v * MD + base];
        float s = 0.f, sb = 0.f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const float x = tmp[v * MD + base + j * st];
          const float bj = fmaf(cw, fabsf(x - c), fmaf(cw64, fabsf(x), ut[v * MD + base + j * st]));
          s = fmaf(L.Dn[i * N + j], x - c, s);
          sb = fmaf(L.Dna[i * N + j], bj, sb);
        }
        acc[v] = fmaf(fabsf(s), W, acc[v]);
        accb[v] = fmaf(sb, W, accb[v]);
      }
    }
  }
  const float r = tile_reduce<DIM, M, N, NV, false>(acc, red, t);
  const float rb = tile_reduce<DIM, M, N, NV, false>(accb, red + NV * MD, t);
  if (t < NS * NV) {
    const int v = t / NS, s = t % NS;
    const float h = float(N) / float(M);
    const float hd = (DIM == 2) ? h : h * h;
    fs[F::sg + v * S + off + s] = hd * r;
    fs[F::eg + v * S + off + s] = 1.01f * hd * rb;
  }
  __syncthreads();
  return sq_all ? 1 : 2;
}

// raw blending factors of level NP from the FP32 sigmas and their bounds, decided
// where certain (0 or 1, written to alpha with the beta_L rule and the threshold-near
// test of the FP64 path); false (CTA-uniform, nothing written) if any stays open
template <int DIM, int M, int NP>
__device__ bool factor_f32(float* fs, const double* beta, double* alpha, const KParams& par, int t, bool& near) {
  using F = F32Scratch<DIM, M>;
  constexpr int NV = F::NV, S = F::S;
  constexpr int NSP = ipow(M / NP, DIM);
  constexpr int kp = M / NP, kc = M / (NP / 2);
  constexpr int offp = s_off(M, DIM, NP), offc = s_off(M, DIM, NP / 2);
  constexpr float kap = float(DIM + ipow(M, DIM) + 8) * 0x1p-24f;
  const float* sg = fs + F::sg;
  const float* eg = fs + F::eg;
  int* code = reinterpret_cast<int*>(fs + F::code);
  if (t < NSP * NV) {
    const int sp_i = t / NV, v = t % NV;
    const int px = sp_i % kp, py = (sp_i / kp) % kp, pz = (DIM == 3) ? sp_i / (kp * kp) : 0;
    float cs = 0.f, ce = 0.f;
    for (int dz = 0; dz < (DIM == 3 ? 2 : 1); ++dz)
      for (int dy = 0; dy < 2; ++dy) {
        const int c0 = 2 * px + kc * (2 * py + dy + kc * (2 * pz + dz));
        cs += sg[v * S + offc + c0] + sg[v * S + offc + c0 + 1];
        ce += eg[v * S + offc + c0] + eg[v * S + offc + c0 + 1];
      }
    const float sp = sg[v * S + offp + sp_i], ep = eg[v * S + offp + sp_i];
    const float num = fabsf(sp - cs), den = fmaxf(fmaxf(sp, cs), 1.f);
    const float dl = 1.01f * (ep + ce + kap * (sp + cs));
    const float hi = (num + dl) / fmaxf(den - dl, 1.f) * (1.f + 8.f * 0x1p-24f);
    const float lo = (num - dl) / (den + dl) * (1.f - 8.f * 0x1p-24f);
    int c = 2;   // open
    if (isfinite(sp) && isfinite(cs) && isfinite(dl) && isfinite(hi)) {
      if (hi < (float)par.tauS * (1.f - 1e-6f)) c = 1;
      else if (lo > (float)(par.tauS + 1.0 / par.tauA) * (1.f + 1e-6f)) c = 0;
    }
    code[t] = c;
  }
  __syncthreads();
  bool open = false;
  double a = 0.0;
  if (t < NSP) {
    bool any0 = false, all1 = true;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int c = code[t * NV + v];
      any0 = any0 || c == 0;
      all1 = all1 && c == 1;
    }
    if (any0) a = 0.0;
    else if (all1) a = 1.0;
    else open = true;
  }
  if (__syncthreads_or(open)) return false;
  if (t < NSP) {
    if (beta[offp + t] < par.betaL) a = 0.0;
    alpha[offp + t] = a;
    near = near || near_threshold(a, beta[offp + t], par);
  }
  __syncthreads();
  return true;
}

// the level loop of the indicator on the FP32 statistics; true when every factor it
// visits was decided and every squeezing it reaches certified to leave beta = 1 (beta
// then stays 1). sqfree: the levels the element-wide range test settled. fs:
// F32Scratch floats.
template <int DIM, int M>
__device__ bool indicator_f32(const double* su, float* fs, const KParams& p, int sqfree, double* alpha, double* beta,
                              double* refd, bool& near, int fam, int t) {
  using F = F32Scratch<DIM, M>;
  constexpr int MD = F::MD, NV = F::NV, NW = F::NW;
  // reference values (the element's first means in FP32, kept in refd as doubles),
  // the deviations from them (formed in FP64, then rounded), and the element maxima
  // of |deviation|
  if (t < NV) {
    const float r = (float)su[t * MD];
    fs[F::ref + t] = r;
    refd[t] = (double)r;
  }
  __syncthreads();
  float aq[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    aq[v] = 0.f;
    if (t < MD) {
      const float dv = (float)(su[v * MD + t] - refd[v]);
      fs[F::sf + v * MD + t] = dv;
      aq[v] = fabsf(dv);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o /= 2)
#pragma unroll
    for (int v = 0; v < NV; ++v) aq[v] = fmaxf(aq[v], __shfl_xor_sync(0xffffffffu, aq[v], o));
  if (t % 32 == 0)
#pragma unroll
    for (int v = 0; v < NV; ++v) fs[F::qw + v * NW + t / 32] = aq[v];
  __syncthreads();
  if (t < NV) {
    float md = 0.f;
    for (int k = 0; k < NW; ++k) md = fmaxf(md, fs[F::qw + t * NW + k]);
    // |d| <= (1 + u) |fl(d)| and |mean| <= |r| + |d|; the FP64 evaluation's share is
    // 2^-28 max |mean|
    fs[F::q + t] = (md + 0x1p-28f * (fabsf(fs[F::ref + t]) + 2.f * md)) * (1.f + 4.f * 0x1p-24f);
  }
  __syncthreads();
  // each level's squeezing is certified where the FP64 evaluation would squeeze it
  // (a level the element-wide range test left open, and that the loop reaches)
  const float g = (float)p.gamma;
  const bool sqM = !(sqfree & (1 << ilog2(M)));
  if (level_sigma_f32<DIM, M, M>(fs, g, fam, sqM, t) != 1) return false;
  bool stopped = false;
  if (M == 8) {
    const int r4 = level_sigma_f32<DIM, M, 4>(fs, g, fam, !(sqfree & (1 << 2)), t);
    if (r4 == 0) return false;
    if (!factor_f32<DIM, M, (M >= 8 ? 8 : 4)>(fs, beta, alpha, p, t, near)) return false;
    stopped = snap<DIM, M, (M >= 8 ? 8 : 4)>(alpha, p.alphaH, p.alphaL, t);
    if (p.single_level) stopped = true;
    if (!stopped && r4 != 1) return false;
  }
  if (!stopped) {
    const int r2 = level_sigma_f32<DIM, M, 2>(fs, g, fam, !(sqfree & (1 << 1)), t);
    if (r2 == 0) return false;
    if (!factor_f32<DIM, M, 4>(fs, beta, alpha, p, t, near)) return false;
    stopped = snap<DIM, M, 4>(alpha, p.alphaH, p.alphaL, t);
    if (!stopped && !p.single_level) {
      if (r2 != 1) return false;
      constexpr int NS2 = ipow(M / 2, DIM);
      constexpr int off2 = s_off(M, DIM, 2);
      if (t < NS2) {
        const double b = beta[off2 + t];
        alpha[off2 + t] = (b < p.betaL) ? 0.0 : b;   // alpha^(2) := beta^(2)
        near = near || near_threshold(alpha[off2 + t], b, p);
      }
      __syncthreads();
      snap<DIM, M, 2>(alpha, p.alphaH, p.alphaL, t);
    }
  }
  return true;
}

// K1 for element e of one problem (u: the problem's state); sm: K1Smem bytes
// Element of CTA b in class order (lists count[16], list[16][E] filled by an indicator
// launch); the identity when there are no lists or they do not hold every element
// exactly once (no launch yet, or one that skipped elements)
__device__ __forceinline__ int class_order(const int* count, const int* list, int E, int b) {
  if (!list) return b;   // uniform: no lists, no barrier
  __shared__ int se;
  if (threadIdx.x == 0) {
    int e = b;
    {
      int cnt[16], tot = 0;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        cnt[c] = count[c];
        tot += cnt[c];
      }
      if (tot == E) {
        int r = b;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          if (r >= 0 && r < cnt[c]) e = list[(size_t)c * E + r];
          r -= cnt[c];
        }
      }
    }
    se = e;
  }
  __syncthreads();
  return se;
}

template <int DIM, int M>
__device__ __forceinline__ void indicator_body(const KParams& p, const double* __restrict__ u,
                                               const double* __restrict__ frozen, const Work& w, const int e_in,
                                               double* sm) {
  const int e = (int)chk(e_in, p.E, w.counters);
  constexpr int MD = Geo<DIM, M>::MD, NV = Geo<DIM, M>::NV, S = Geo<DIM, M>::S, NL = Geo<DIM, M>::NL;
  constexpr int P = Geo<DIM, M>::P, NT = Geo<DIM, M>::NT;
  using L = K1Smem<DIM, M>;
  double* alpha = sm + L::d_alpha;
  double* beta = sm + L::d_beta;
  double* brho = sm + L::d_brho;
  double* redd = sm + L::d_red;
  double* epsv = sm + L::d_eps;
  real* rs = reinterpret_cast<real*>(sm + L::d_total);
  real* su = rs + L::r_su;
  real* ut = rs + L::r_ut;
  real* tmp = rs + L::r_tmp;
  real* red = rs + L::r_red;
  real* th = rs + L::r_th;
  real* avg = rs + L::r_avg;
  real* sig = rs + L::r_sig;
  real* alf = rs + L::r_alf;
  real* bef = rs + L::r_bef;
  const int t = threadIdx.x;
  const real g = (real)p.gamma;
  const int fam = p.family;
  const double* ue = u + (size_t)e * NV * MD;
  // FP64 build: the element's means by one bulk copy into su. The FP32 build converts
  // them on the way in with plain loads (a copy into scratch and a conversion pass
  // from there measured 2-4 % slower: nothing here overlaps the copy)
  __shared__ unsigned long long stage_bar;
  constexpr unsigned SB = NV * MD * sizeof(double);
  const bool bulk = sizeof(real) == 8 && stage_ok(ue, su, SB);
  __syncthreads();
  if (bulk) stage_issue(&stage_bar, su, ue, SB);
  for (int i = t; i < S; i += NT) { alpha[i] = 0.0; beta[i] = 1.0; }
  if (bulk) {
    if (!stage_wait(&stage_bar, &w.counters[0], p.stage_cap)) return;
  } else {
    for (int i = t; i < NV * MD; i += NT) su[i] = (real)ue[i];
  }
  __syncthreads();
  // non-permissible mean values (rho <= 0 or 2 rho E <= |m|^2)
  if (t < MD) {
    real q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = su[v * MD + t];
    if (!permissible64<DIM>(q)) atomicOr((unsigned long long*)&w.counters[0], 1ull);
  }
  if (frozen != nullptr) {
    const double* fe = frozen + (size_t)e * 2 * S;
    for (int i = t; i < S; i += NT) { alpha[i] = fe[i]; beta[i] = fe[S + i]; }
    sub_averages<DIM, M, 2>(su, red, avg, t);
    sub_averages<DIM, M, 4>(su, red, avg, t);
    if (M == 8) sub_averages<DIM, M, (M >= 8 ? 8 : 4)>(su, red, avg, t);
  } else {
    bool near = false;
    bool settled = false;
    if constexpr (sizeof(real) == 8) {
      // the certified FP32 pass decides the element's levels where it can, certifying
      // every squeezing it reaches; otherwise the FP64 evaluation below runs from the
      // start (with the element-wide range test of the squeezing)
      static_assert(F32Scratch<DIM, M>::total * sizeof(float) <= (L::r_total - L::r_ut) * sizeof(real),
                    "FP32 pass scratch exceeds the indicator's shared memory");
      if (p.fp32_filter) {
        settled = indicator_f32<DIM, M>(reinterpret_cast<const double*>(su), reinterpret_cast<float*>(ut), p, 0,
                                        alpha, beta, redd, near, fam, t);
        if (settled) {
          if (t == 0) atomicAdd((unsigned long long*)&w.counters[12], 1ull);
        } else {
          near = false;
          for (int i = t; i < S; i += NT) { alpha[i] = 0.0; beta[i] = 1.0; }
          __syncthreads();
        }
      }
    }
    if (!settled) {
      const int sqfree = squeeze_free_levels<DIM, M>(su, rs + L::r_bnd, g, fam, t);
      level_stats<DIM, M, M>(su, ut, tmp, red, avg, sig, g, fam, t);
      if (!(sqfree & (1 << ilog2(M)))) squeeze<DIM, M, M>(su, ut, red, avg, beta, brho, epsv, p.gamma, fam, t, w.counters);
      bool stopped = false;
      if (M == 8) {
        level_stats<DIM, M, 4>(su, ut, tmp, red, avg, sig, g, fam, t);
        blending_factor<DIM, M, (M >= 8 ? 8 : 4)>(sig, beta, alpha, redd, p.tauA, p.tauS, p.betaL, t, p, near);
        stopped = snap<DIM, M, (M >= 8 ? 8 : 4)>(alpha, p.alphaH, p.alphaL, t);
        if (p.single_level) stopped = true;   // single-level scheme: levels below M stay off
        if (!stopped && !(sqfree & (1 << 2)))
          squeeze<DIM, M, 4>(su, ut, red, avg, beta, brho, epsv, p.gamma, fam, t, w.counters);
      }
      if (!stopped) {
        level_stats<DIM, M, 2>(su, ut, tmp, red, avg, sig, g, fam, t);
        blending_factor<DIM, M, 4>(sig, beta, alpha, redd, p.tauA, p.tauS, p.betaL, t, p, near);
        stopped = snap<DIM, M, 4>(alpha, p.alphaH, p.alphaL, t);
        if (!stopped && !p.single_level) {
          if (!(sqfree & (1 << 1))) squeeze<DIM, M, 2>(su, ut, red, avg, beta, brho, epsv, p.gamma, fam, t, w.counters);
          constexpr int NS2 = ipow(M / 2, DIM);
          constexpr int off2 = s_off(M, DIM, 2);
          if (t < NS2) {
            const double b = beta[off2 + t];
            alpha[off2 + t] = (b < p.betaL) ? 0.0 : b;   // alpha^(2) := beta^(2)
            near = near || near_threshold(alpha[off2 + t], b, p);
          }
          __syncthreads();
          snap<DIM, M, 2>(alpha, p.alphaH, p.alphaL, t);
        }
      }
    }
    if (__syncthreads_or(near) && t == 0) atomicAdd((unsigned long long*)&w.counters[3], 1ull);
  }
  __syncthreads();
  for (int i = t; i < S; i += NT) { alf[i] = (real)alpha[i]; bef[i] = (real)beta[i]; }
  __syncthreads();
  // blending weights per subcell (eq. blending-weights) in the compute type; in FP64
  // a snapped factor (0 or 1, recognised from its bits on the integer units) needs no
  // FP64 arithmetic: A rest and rest (1 - A) are then exact
  if (t < MD) {
    real rest = 1;
#pragma unroll
    for (int l = NL - 1; l >= 1; --l) {
      const int n = 1 << l;
      const real A = alf[s_off(M, DIM, n) + sub_index<DIM, M>(t, n)];
      if constexpr (sizeof(real) == 8) {
        const long long bits = __double_as_longlong(A);
        if (bits == 0ll) {
          th[l * MD + t] = real(0);
          continue;
        }
        if (bits == 0x3FF0000000000000ll) {
          th[l * MD + t] = rest;
          rest = real(0);
          continue;
        }
      }
      th[l * MD + t] = A * rest;
      rest = rest * (real(1) - A);
    }
    th[t] = rest;
  }
  __syncthreads();
  // level bounds of the element (FP64: a nonzero weight by its bits, sign ignored)
  int used = 0;
#pragma unroll
  for (int l = 0; l < NL; ++l) {
    bool nz = false;
    if (t < MD) {
      if constexpr (sizeof(real) == 8) nz = (__double_as_longlong(th[l * MD + t]) << 1) != 0ll;
      else nz = th[l * MD + t] != real(0);
    }
    used |= __syncthreads_or(nz) ? (1 << l) : 0;
  }
  if (t == 0) {
    int lo = 0, hi = 0;
    for (int l = 0; l < NL; ++l)
      if (used & (1 << l)) { lo = l; break; }
    for (int l = NL - 1; l >= 0; --l)
      if (used & (1 << l)) { hi = l; break; }
    w.decision[e] = (uint8_t)(lo | (hi << 4));
    if (w.class_list) {   // (a launch without the count reset overflows: the lists are then ignored)
      const int pos = atomicAdd(&w.class_count[used], 1);
      if (pos < p.E) w.class_list[(size_t)used * p.E + pos] = e;
    }
    atomicAdd((unsigned long long*)&w.counters[4 + lo], 1ull);
    atomicAdd((unsigned long long*)&w.counters[8 + hi], 1ull);
    atomicAdd((unsigned long long*)&w.counters[16 + used], 1ull);
  }
  double* ce = w.coeffs + (size_t)e * 2 * S;
  for (int i = t; i < S; i += NT) { ce[i] = alpha[i]; ce[S + i] = beta[i]; }
  // blended states of the element faces and their weights
  real* fstates = reinterpret_cast<real*>(w.face_states);
  for (int i = t; i < 2 * DIM * P; i += NT) {
    const int face = i / P, j = i % P, a = face / 2, side = face % 2;
    const int tt = subcell_of<DIM, M>(a, side ? M - 1 : 0, j);
    real Ub[NV];
    blended_face_state<DIM, M>(su, th, bef, avg, tt, a, side, fam, Ub);
    real* fs = fstates + ((size_t)e * 2 * DIM + face) * (NV + NL) * P;
#pragma unroll
    for (int v = 0; v < NV; ++v) fs[v * P + j] = Ub[v];
#pragma unroll
    for (int l = 0; l < NL; ++l) fs[(NV + l) * P + j] = th[l * MD + tt];
  }
}

// resident CTAs per SM requested for the indicator kernel: caps at the register
// counts the compiler chose without a bound (an explicit bound of 1 let it take more
// and halved the occupancy in 3D), except 2D M = 8 in the FP32 build, where 24 CTAs of
// 64 threads (40 registers) measured faster than the unbounded 56 registers
template <int DIM, int M>
struct K1MinBlocks {
  static constexpr int v = sizeof(real) == 8 ? (DIM == 2 ? (M == 4 ? 21 : 12) : (M == 4 ? 10 : 1))
                                             : (DIM == 2 ? (M == 4 ? 32 : 24) : (M == 4 ? 16 : 2));
};

template <int DIM, int M>
__global__ void __launch_bounds__(Geo<DIM, M>::NT, K1MinBlocks<DIM, M>::v)
    k_indicator(KParams p, const double* __restrict__ u, const double* __restrict__ frozen, Work w) {
  extern __shared__ double sm[];
  indicator_body<DIM, M>(p, u, frozen, w, w.order ? w.order[blockIdx.x] : (int)blockIdx.x, sm);
}

// ---------------------------------------------------------------------------
// K2: interface fluxes at element faces
// ---------------------------------------------------------------------------
template <int DIM, int M>
struct FaceCfg {
  static constexpr int P = Geo<DIM, M>::P;
  static constexpr int NT = 128;
  static constexpr int NF = NT / P;   // faces per CTA
};

// shared scratch of one face group of NF faces: sUL, sUR, sT, sF (NF NV P reals
// each) and sflag (NF P ints)
template <int DIM, int M, int NF>
struct FaceSmem {
  static constexpr int NV = Geo<DIM, M>::NV, P = Geo<DIM, M>::P;
  static constexpr size_t bytes = sizeof(real) * 4 * NF * NV * P + sizeof(int) * NF * P;
};

// K2 for the NF faces fid0 ... fid0 + NF - 1 of direction a of one problem (threads
// tid < NF P; a block of more threads leaves the rest idle); scratch: FaceSmem
template <int DIM, int M, int NF>
__device__ __forceinline__ void face_body_s(const KParams& p, const Work& w, int a, int nfaces, int fid0,
                                           unsigned char* scratch) {
  constexpr int NV = Geo<DIM, M>::NV, NL = Geo<DIM, M>::NL, P = Geo<DIM, M>::P;
  real* sUL = reinterpret_cast<real*>(scratch);
  real* sUR = sUL + NF * NV * P;
  real* sT = sUR + NF * NV * P;
  real* sF = sT + NF * NV * P;
  int* sflag = reinterpret_cast<int*>(sF + NF * NV * P);
  const int tid = threadIdx.x < NF * P ? threadIdx.x : NF * P;
  const int f = tid < NF * P ? tid / P : 0, j = tid % P;
  const int fid = fid0 + f;
  const bool valid = tid < NF * P && fid < nfaces;
  const real* fstates = reinterpret_cast<const real*>(w.face_states);
  real UL[NV], UR[NV], wl[NL];
  if (valid) {
    const int NA = p.nfaces_along[a];
    const int fa = fid % NA, tr = fid / NA;
    const bool periodic = p.bc[2 * a] == 0;
    const int na = p.nel[a];
    int eL = fa - 1, eR = fa;
    if (periodic && eL < 0) eL = na - 1;
    const bool ghostL = !periodic && fa == 0;
    const bool ghostR = !periodic && fa == na;
    auto elin = [&](int ea) { return chk(element_of<DIM>(p, a, ea, tr), p.E, w.counters); };
    const size_t fsz = (size_t)(NV + NL) * P;
    real thL[NL], thR[NL];
    if (!ghostL) {
      const real* fsL = fstates + ((size_t)elin(eL) * 2 * DIM + 2 * a + 1) * fsz;
      for (int v = 0; v < NV; ++v) UL[v] = fsL[v * P + j];
      for (int l = 0; l < NL; ++l) thL[l] = fsL[(NV + l) * P + j];
    }
    if (!ghostR) {
      const real* fsR = fstates + ((size_t)elin(eR) * 2 * DIM + 2 * a + 0) * fsz;
      for (int v = 0; v < NV; ++v) UR[v] = fsR[v * P + j];
      for (int l = 0; l < NL; ++l) thR[l] = fsR[(NV + l) * P + j];
    }
    if (ghostL && p.bc[2 * a] == SESC_BC_HALO) {
      // partition side: the neighbouring part's face states of this face (its high
      // side), received into the halo buffer, row tr
      const real* hs = reinterpret_cast<const real*>(w.halo[2 * a]) + (size_t)chk(tr, p.E / na, w.counters) * fsz;
      for (int v = 0; v < NV; ++v) UL[v] = hs[v * P + j];
      for (int l = 0; l < NL; ++l) thL[l] = hs[(NV + l) * P + j];
    } else if (ghostL) {   // low boundary: ghost from the right state (reading R6)
      for (int v = 0; v < NV; ++v) UL[v] = UR[v];
      if (p.bc[2 * a] == 1)
#pragma unroll
        for (int k = 0; k < DIM; ++k)
          if (a == k) UL[1 + k] = -UL[1 + k];
      for (int l = 0; l < NL; ++l) thL[l] = thR[l];
    }
    if (ghostR && p.bc[2 * a + 1] == SESC_BC_HALO) {
      const real* hs = reinterpret_cast<const real*>(w.halo[2 * a + 1]) + (size_t)chk(tr, p.E / na, w.counters) * fsz;
      for (int v = 0; v < NV; ++v) UR[v] = hs[v * P + j];
      for (int l = 0; l < NL; ++l) thR[l] = hs[(NV + l) * P + j];
    } else if (ghostR) {
      for (int v = 0; v < NV; ++v) UR[v] = UL[v];
      if (p.bc[2 * a + 1] == 1)
#pragma unroll
        for (int k = 0; k < DIM; ++k)
          if (a == k) UR[1 + k] = -UR[1 + k];
      for (int l = 0; l < NL; ++l) thR[l] = thL[l];
    }
    for (int l = 0; l < NL; ++l) wl[l] = real(0.5) * (thL[l] + thR[l]);
  } else {
    for (int v = 0; v < NV; ++v) { UL[v] = 1; UR[v] = 1; }
    for (int l = 0; l < NL; ++l) wl[l] = 0;
  }
  real F[NV];
  blended_flux<DIM, M>(UL, UR, wl, a, (real)p.gamma, p.family, f, j, valid, sUL, sUR, sT, sF, sflag, F, w.counters);
  if (valid) {   // stored in FP64: K3 takes its flux differences at element faces from these
    double* out = w.face_flux + (size_t)chk((long long)p.face_off[a] + fid, p.nfaces, w.counters) * NV * P;
    for (int v = 0; v < NV; ++v) out[v * P + j] = (double)F[v];
  }
}

template <int DIM, int M>
__device__ __forceinline__ void face_body(const KParams& p, const Work& w, int a, int nfaces, int fid0) {
  constexpr int NF = FaceCfg<DIM, M>::NF;
  __shared__ __align__(16) unsigned char scratch[FaceSmem<DIM, M, NF>::bytes];
  face_body_s<DIM, M, NF>(p, w, a, nfaces, fid0, scratch);
}

template <int DIM, int M>
__global__ void __launch_bounds__(128) k_face_flux(KParams p, Work w, int a, int nfaces) {
  face_body<DIM, M>(p, w, a, nfaces, blockIdx.x * FaceCfg<DIM, M>::NF);
}

// The element-face states (blended states and level weights, the data a partition
// exchanges: appendix 3D extension, face-centred means and blending factors) of the
// face `side` (0 low, 1 high) along a of the boundary layer of elements on that side,
// packed row by row (transverse element index tr as in K2) into dst[tr][nv + L][P].
template <int DIM, int M>
__global__ void k_pack_halo(KParams p, Work w, int a, int side, real* __restrict__ dst, int ntr) {
  constexpr int NV = Geo<DIM, M>::NV, NL = Geo<DIM, M>::NL, P = Geo<DIM, M>::P;
  constexpr int FS = (NV + NL) * P;
  const real* fstates = reinterpret_cast<const real*>(w.face_states);
  const size_t n = (size_t)ntr * FS;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int tr = (int)(i / FS), r = (int)(i % FS);
    const size_t e = (size_t)chk(element_of<DIM>(p, a, side ? p.nel[a] - 1 : 0, tr), p.E, w.counters);
    dst[i] = fstates[(e * 2 * DIM + 2 * a + side) * FS + r];
  }
}

// ---------------------------------------------------------------------------
// K3: level right-hand sides in subcell-flux form, blend, RK stage
// ---------------------------------------------------------------------------
template <int DIM, int M>
struct K3Smem {
  static constexpr int MD = Geo<DIM, M>::MD, NV = Geo<DIM, M>::NV, S = Geo<DIM, M>::S, NL = Geo<DIM, M>::NL;
  static constexpr int P = Geo<DIM, M>::P;
  static constexpr int FB = (M - 1) * NV * P;   // one face-group buffer
  static constexpr int d_alpha = 0;
  static constexpr int d_beta = d_alpha + S;
  static constexpr int d_gd = d_beta + S;            // interior subcell fluxes of one level and direction, FP64
  // element face fluxes in FP64 (the FP64 build reads them from the compute-type array)
  static constexpr int d_fb64 = d_gd + NV * MD;
  static constexpr int d_total = d_fb64 + (sizeof(real) == 4 ? 2 * DIM * NV * P : 0);
  static constexpr int r_su = 0;
  static constexpr int r_th = r_su + NV * MD;
  static constexpr int r_avg = r_th + NL * MD;
  static constexpr int r_fb = r_avg + NV * S;                 // element face fluxes [2 DIM][NV][P]
  static constexpr int r_fin = r_fb + 2 * DIM * NV * P;      // inner interface fluxes of every direction
  static constexpr int r_bef = r_fin + DIM * FB;             // beta in the compute type
  static constexpr int r_u = r_bef + S;                      // union: face scratch (4 FB) | level scratch (3 NV MD)
  static constexpr int uni = (4 * FB > 3 * NV * MD ? 4 * FB : 3 * NV * MD);
  static constexpr int r_total = r_u + uni;
  static constexpr int i_flag = (M - 1) * P;
  static constexpr size_t bytes = sizeof(double) * d_total + sizeof(real) * r_total + sizeof(int) * i_flag;
};

// beta-limited nodal values of level N in ut (eq. positivity-limiter-applied)
template <int DIM, int M, int N>
__device__ void limited_nodal(const real* su, const real* avg, const real* beta, real* ut, real* tmp,
                              const KParams& p, int t) {
  constexpr int MD = ipow(M, DIM), NV = DIM + 2, S = Geo<DIM, M>::S;
  constexpr int off = s_off(M, DIM, N);
  reconstruct<DIM, M, N>(ut, tmp, su, p.family, t);
  if (t < MD) {
    const int s = sub_index<DIM, M>(t, N);
    const real b = beta[off + s];
    if (b != real(1)) {
#pragma unroll
      for (int v = 0; v < NV; ++v) ut[v * MD + t] = (real(1) - b) * avg[v * S + off + s] + b * ut[v * MD + t];
    }
  }
  __syncthreads();
}

// interior subcell fluxes of level N along a (telescoping form, see opgen.h):
// G_k = c0_k F_L + cn_k F_R - (1/N) (f x_a C x_b P)_k for k = 1..N-1 of every
// sub-element, stored at the subcell left of the interface; then every subcell
// adds theta * (M/dx) * (G_right - G_left) to its FP64 accumulator.
template <int DIM, int M, int N>
__device__ void level_fluxes(const real* ut, real* tmp, real* fb, const real* fbd, const double* fb64,
                             const real* fin, double* gd, const KParams& p, int a, int t, bool thc_on, double thc,
                             double* acc) {
  constexpr int MD = ipow(M, DIM), NV = DIM + 2, P = ipow(M, DIM - 1);
  const DevLevel& L = lev(p.family, ilog2(N));
  // nodal fluxes in direction a (the primitives are formed again per direction: kept
  // across the direction loop they cost more registers than the division they save)
  if (t < MD) {
    real q[NV], f[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = ut[v * MD + t];
    Prim<DIM> w;
    w.load(q, (real)p.gamma);
    flux_of<DIM>(q, w, a, f);
#pragma unroll
    for (int v = 0; v < NV; ++v) fb[v * MD + t] = f[v];
  }
  __syncthreads();
  // cumulative volume operator along a: output k = i + 1 at local index i < N - 1
  if (t < MD) {
    const int st = stride_of<M>(a);
    const int i = coord_of<M>(t, a) % N, base = t - i * st;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      real s = 0;
      if (i < N - 1) {
#pragma unroll
        for (int j = 0; j < N; ++j) s = fma(L.C[i * N + j], fb[v * MD + base + j * st], s);
      }
      tmp[v * MD + t] = s;
    }
  }
  __syncthreads();
  real* src = tmp;
  real* dst = fb;
#pragma unroll
  for (int b = 0; b < DIM; ++b) {
    if (b == a) continue;
    mode_sq<DIM, M, N, NV>(dst, src, L.P, b, t);
    __syncthreads();
    real* x = src;
    src = dst;
    dst = x;
  }
  // src holds W; G at the subcell left of each interior interface
  const bool act = t < MD;
  const int c = act ? coord_of<M>(t, a) : 0;
  const int i = c % N, lo = c - i;
  int j = 0;
  if (DIM == 2) j = (a == 0) ? (t / M) : (t % M);
  else {
    const int cx = t % M, cy = (t / M) % M, cz = t / (M * M);
    j = (a == 0) ? (cy + M * cz) : (a == 1 ? (cx + M * cz) : (cx + M * cy));
  }
  auto flux_at = [&](int k, int v) -> real {
    if (k == 0) return fbd[((2 * a + 0) * NV + v) * P + j];
    if (k == M) return fbd[((2 * a + 1) * NV + v) * P + j];
    return fin[((k - 1) * NV + v) * P + j];
  };
  // every inner interface value is converted to FP64 once, by the subcell left of
  // it: the level's own flux inside a sub-element, the blended interface flux on a
  // sub-element boundary; element faces come in FP64 (fb64). Both subcells an
  // interface separates read the same FP64 value (conservation to FP64 roundoff).
  if (act && c < M - 1) {
    const real c0 = L.c0[i], cn = L.cn[i], inv = real(1) / real(N);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const real gv = (i < N - 1) ? c0 * flux_at(lo, v) + cn * flux_at(lo + N, v) - inv * src[v * MD + t]
                                  : fin[(c * NV + v) * P + j];
      gd[v * MD + t] = (double)gv;
    }
  }
  __syncthreads();
  if (act && thc_on) {
    const int st = stride_of<M>(a);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double gr = (c == M - 1) ? fb64[((2 * a + 1) * NV + v) * P + j] : gd[v * MD + t];
      const double gl = (c == 0) ? fb64[((2 * a + 0) * NV + v) * P + j] : gd[v * MD + t - st];
      acc[v] = fma(thc, gr - gl, acc[v]);
    }
  }
  __syncthreads();
}

// resident CTAs per SM requested from the register allocator for the update kernel
// in the FP32 build (it is latency-bound there; the FP64 build is FP64-pipe-bound)
template <int DIM, int M>
struct K3MinBlocks {
  static constexpr int v = sizeof(real) == 8 ? (DIM == 2 ? 6 : 1) : (DIM == 2 ? (M == 4 ? 24 : 16) : (M == 4 ? 10 : 1));
};

// K3 for element e of one problem; sm: K3Smem bytes
template <int DIM, int M>
__device__ __forceinline__ void update_body(const KParams& p, const Work& w, const double* __restrict__ us,
                                            const double* __restrict__ u0, double* __restrict__ out, double ark,
                                            double brk, double dt, const double* dt_dev, int mode, const int e_in,
                                            double* sm, const StageTerm& x) {
  const int e = (int)chk(e_in, p.E, w.counters);
  constexpr int MD = Geo<DIM, M>::MD, NV = Geo<DIM, M>::NV, S = Geo<DIM, M>::S, NL = Geo<DIM, M>::NL;
  constexpr int P = Geo<DIM, M>::P, NT = Geo<DIM, M>::NT;
  using L = K3Smem<DIM, M>;
  double* alpha = sm + L::d_alpha;
  double* beta = sm + L::d_beta;
  double* gd = sm + L::d_gd;
  real* rs = reinterpret_cast<real*>(sm + L::d_total);
  real* su = rs + L::r_su;
  real* th = rs + L::r_th;
  real* avg = rs + L::r_avg;
  real* fbd = rs + L::r_fb;
  real* fin = rs + L::r_fin;
  real* bef = rs + L::r_bef;
  real* uni = rs + L::r_u;
  int* sflag = reinterpret_cast<int*>(rs + L::r_total);
  const int t = threadIdx.x;
  const int fam = p.family;
  const real g = (real)p.gamma;
  const double* ue = us + (size_t)e * NV * MD;
  // the element's means by one bulk copy, in flight while the coefficients and the
  // element face fluxes load: into su (FP64 build) or into the (16-byte aligned)
  // union scratch and converted from there (FP32 build)
  static_assert(3 * NV * MD >= 2 * NV * MD + 3, "staging area");
  __shared__ unsigned long long stage_bar;
  double* stg = (sizeof(real) == 8)
                    ? reinterpret_cast<double*>(su)
                    : reinterpret_cast<double*>(uni + ((16u - (smem_u32(uni) & 15u)) & 15u) / sizeof(real));
  constexpr unsigned SB = NV * MD * sizeof(double);
  const bool bulk = stage_ok(ue, stg, SB);
  __syncthreads();
  if (bulk) stage_issue(&stage_bar, stg, ue, SB);
  else
    for (int i = t; i < NV * MD; i += NT) su[i] = (real)ue[i];
  const double* ce = w.coeffs + (size_t)e * 2 * S;
  for (int i = t; i < S; i += NT) {
    alpha[i] = ce[i];
    beta[i] = ce[S + i];
    bef[i] = (real)ce[S + i];
  }
  int ec[3];
  ec[0] = e % p.nel[0];
  ec[1] = (e / p.nel[0]) % p.nel[1];
  ec[2] = (DIM == 3) ? e / (p.nel[0] * p.nel[1]) : 0;
  // element face fluxes (FP64 in memory; the compute-type copy feeds the level fluxes)
  double* fb64 = (sizeof(real) == 8) ? reinterpret_cast<double*>(fbd) : sm + L::d_fb64;
  const double* fflux = w.face_flux;
  for (int i = t; i < 2 * DIM * NV * P; i += NT) {
    const int face = i / (NV * P), r = i % (NV * P);
    const int a = face / 2, side = face % 2;
    const int NA = p.nfaces_along[a];
    int fa = pick(ec, a) + side;
    if (p.bc[2 * a] == 0 && fa == p.nel[a]) fa = 0;
    int tr;
    if (DIM == 2) tr = pick(ec, 1 - a);
    else tr = (a == 0) ? ec[1] + p.nel[1] * ec[2] : (a == 1 ? ec[0] + p.nel[0] * ec[2] : ec[0] + p.nel[0] * ec[1]);
    const size_t fid = (size_t)chk((long long)p.face_off[a] + fa + (long long)NA * tr, p.nfaces, w.counters);
    const double fv = fflux[fid * NV * P + r];
    fb64[i] = fv;
    fbd[i] = (real)fv;
  }
  if (bulk) {
    if (!stage_wait(&stage_bar, &w.counters[0], p.stage_cap)) return;
    if (sizeof(real) == 4)
      for (int i = t; i < NV * MD; i += NT) su[i] = (real)stg[i];
  }
  __syncthreads();
  // blending weights: FP64 per thread for the flux-difference factors, and in the
  // compute type (same zero pattern) for face states and level tests
  double thv[NL];
  if (t < MD) {
    weights_of<DIM, M>(alpha, t, thv);
    real rest = 1;
#pragma unroll
    for (int l = NL - 1; l >= 1; --l) {
      const int n = 1 << l;
      const real A = (real)alpha[s_off(M, DIM, n) + sub_index<DIM, M>(t, n)];
      th[l * MD + t] = A * rest;
      rest = rest * (real(1) - A);
    }
    th[t] = rest;
  } else {
#pragma unroll
    for (int l = 0; l < NL; ++l) thv[l] = 0.0;
  }
  __syncthreads();
  // levels carrying weight, inner interfaces they use (all for the FV level, the
  // sub-element boundaries for a DG level below M), averages where squeezing acts
  int used = 0;
#pragma unroll
  for (int l = 0; l < NL; ++l) used |= __syncthreads_or(t < MD && th[l * MD + t] != real(0)) ? (1 << l) : 0;
  int kmask = (used & 1) ? ((1 << M) - 2) : 0;
#pragma unroll
  for (int l = 1; l < NL - 1; ++l)
    if (used & (1 << l))
      for (int k = 1 << l; k < M; k += 1 << l) kmask |= 1 << k;
  const int nk = __popc(kmask);
#pragma unroll
  for (int l = 1; l < NL; ++l) {
    if (!(used & (1 << l))) continue;
    const int n = 1 << l;
    const int NS = ipow(M / n, DIM);
    const int off = s_off(M, DIM, n);
    if (!__syncthreads_or(t < NS && bef[off + t] != real(1))) continue;
    if (n == 2) sub_averages<DIM, M, 2>(su, uni, avg, t);
    else if (n == 4) sub_averages<DIM, M, 4>(su, uni, avg, t);
    else sub_averages<DIM, M, (M >= 8 ? 8 : 4)>(su, uni, avg, t);
  }
  __syncthreads();
  constexpr int FB = K3Smem<DIM, M>::FB;
  // inner interface fluxes of every direction: dpp directions side by side per pass
  // (face slot (a mod dpp) nk + f), as many as fit the face buffers and the block
  const int dpp = nk == 0 ? 1 : min(DIM, min((M - 1) / nk, NT / (nk * P)));
#pragma unroll 1   // kept rolled: one copy of the (large) interface-flux code for all directions
  for (int a0 = 0; a0 < DIM; a0 += dpp) {
    if (nk == 0) break;
    real* sUL = uni;
    real* sUR = uni + FB;
    real* sT = uni + 2 * FB;
    real* sF = uni + 3 * FB;
    const bool valid = t < dpp * nk * P && a0 + t / (nk * P) < DIM;
    const int slot = valid ? t / P : 0, j = valid ? t % P : 0;
    const int a = a0 + slot / nk, f = slot % nk;
    int k = 0;
    for (int cnt = -1; cnt < f && k < M - 1;) {
      ++k;
      if (kmask & (1 << k)) ++cnt;
    }
    real UL[NV], UR[NV], wl[NL];
    if (valid) {   // interface k lies between subcells k-1 and k along a
      const int tL = subcell_of<DIM, M>(a, k - 1, j);
      const int tR = tL + stride_of<M>(a);
      if (p.single_level) {   // single-level scheme: inner interfaces take the raw subcell means
#pragma unroll
        for (int v = 0; v < NV; ++v) { UL[v] = su[v * MD + tL]; UR[v] = su[v * MD + tR]; }
#pragma unroll
        for (int l = 0; l < NL; ++l) wl[l] = (l == 0) ? real(1) : real(0);
      } else {
        blended_face_state<DIM, M>(su, th, bef, avg, tL, a, 1, fam, UL);
        blended_face_state<DIM, M>(su, th, bef, avg, tR, a, 0, fam, UR);
#pragma unroll
        for (int l = 0; l < NL; ++l) wl[l] = real(0.5) * (th[l * MD + tL] + th[l * MD + tR]);
      }
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) { UL[v] = 1; UR[v] = 1; }
#pragma unroll
      for (int l = 0; l < NL; ++l) wl[l] = 0;
    }
    real F[NV];
    blended_flux<DIM, M>(UL, UR, wl, a, g, fam, slot, j, valid, sUL, sUR, sT, sF, sflag, F, w.counters);
    if (valid) {
#pragma unroll
      for (int v = 0; v < NV; ++v) fin[a * FB + ((k - 1) * NV + v) * P + j] = F[v];
    }
    __syncthreads();
  }
  double acc[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) acc[v] = 0.0;
  // FV level: theta^(1) (M/dx) (F_right - F_left), FP64; each inner interface flux
  // is converted once (by the subcell left of it) into gd
  if (used & 1) {
#pragma unroll 1
    for (int a = 0; a < DIM; ++a) {
      const bool act = t < MD;
      const int c = act ? coord_of<M>(t, a) : 0;
      int j = 0;
      if (DIM == 2) j = (a == 0) ? (t / M) : (t % M);
      else {
        const int cx = t % M, cy = (t / M) % M, cz = t / (M * M);
        j = (a == 0) ? (cy + M * cz) : (a == 1 ? (cx + M * cz) : (cx + M * cy));
      }
      const real* fa = fin + a * FB;
      if (act && c < M - 1) {
#pragma unroll
        for (int v = 0; v < NV; ++v) gd[v * MD + t] = (double)fa[(c * NV + v) * P + j];
      }
      __syncthreads();
      if (act && th[t] != real(0)) {
        const double thc = p.mdx[a] * thv[0];
        const int st = stride_of<M>(a);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const double fr = (c == M - 1) ? fb64[((2 * a + 1) * NV + v) * P + j] : gd[v * MD + t];
          const double fl = (c == 0) ? fb64[((2 * a + 0) * NV + v) * P + j] : gd[v * MD + t - st];
          acc[v] = fma(thc, fr - fl, acc[v]);
        }
      }
      __syncthreads();
    }
  }
  // DG levels: reconstruct and limit once, then the subcell fluxes along every direction
  {
    real* ut = uni;
    real* tmp = uni + NV * MD;
    real* fb = uni + 2 * NV * MD;
#pragma unroll
    for (int l = 1; l < NL; ++l) {
      if (!(used & (1 << l))) continue;
      if (l == 1) limited_nodal<DIM, M, 2>(su, avg, bef, ut, tmp, p, t);
      else if (l == 2) limited_nodal<DIM, M, 4>(su, avg, bef, ut, tmp, p, t);
      else limited_nodal<DIM, M, (M >= 8 ? 8 : 4)>(su, avg, bef, ut, tmp, p, t);
      const bool on = t < MD && th[l * MD + t] != real(0);
#pragma unroll
      for (int a = 0; a < DIM; ++a) {
        const double thc = on ? p.mdx[a] * thv[l] : 0.0;
        if (l == 1) level_fluxes<DIM, M, 2>(ut, tmp, fb, fbd, fb64, fin + a * FB, gd, p, a, t, on, thc, acc);
        else if (l == 2) level_fluxes<DIM, M, 4>(ut, tmp, fb, fbd, fb64, fin + a * FB, gd, p, a, t, on, thc, acc);
        else
          level_fluxes<DIM, M, (M >= 8 ? 8 : 4)>(ut, tmp, fb, fbd, fb64, fin + a * FB, gd, p, a, t, on, thc, acc);
      }
    }
  }
  if (t < MD) {
    double* oe = out + (size_t)e * NV * MD;
    if (mode == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) oe[v * MD + t] = acc[v];
    } else {
      const double dtv = x.g * (dt_dev ? *dt_dev : dt);   // x.g = 1 for the two-term stages
      const double* u0e = u0 + (size_t)e * NV * MD;
      const double* u2e = x.u2 ? x.u2 + (size_t)e * NV * MD : nullptr;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        // the FP64 build's su is the stage state itself
        const double r = fma(dtv, acc[v], sizeof(real) == 8 ? (double)su[v * MD + t] : ue[v * MD + t]);
        double o;
        if (ark == 0.0) o = (brk == 1.0) ? r : brk * r;
        else o = fma(ark, u0e[v * MD + t], brk * r);
        if (u2e) o = fma(x.c, u2e[v * MD + t], o);
        oe[v * MD + t] = o;
      }
    }
  }
}


template <int DIM, int M>
__global__ void __launch_bounds__(Geo<DIM, M>::NT, K3MinBlocks<DIM, M>::v)
    k_update(KParams p, Work w, const double* __restrict__ us, const double* __restrict__ u0, double* __restrict__ out,
             double ark, double brk, double dt, const double* dt_dev, int mode, StageTerm x) {
  extern __shared__ double sm[];
  const int e = class_order(w.class_count, w.class_list, p.E, blockIdx.x);
  if (w.order && threadIdx.x == 0) w.order[blockIdx.x] = e;
  update_body<DIM, M>(p, w, us, u0, out, ark, brk, dt, dt_dev, mode, e, sm, x);
}

// ---------------------------------------------------------------------------
// theta / abar output of sesc_indicator
// ---------------------------------------------------------------------------
template <int DIM, int M>
__global__ void k_theta(KParams p, Work w, double* theta, double* abar) {
  constexpr int MD = Geo<DIM, M>::MD, S = Geo<DIM, M>::S, NL = Geo<DIM, M>::NL;
  const int e = blockIdx.x, t = threadIdx.x;
  if (t >= MD) return;
  const double* ce = w.coeffs + (size_t)e * 2 * S;
  double thl[NL];
  weights_of<DIM, M>(ce, t, thl);
  if (theta) {
    for (int l = 0; l < NL; ++l) theta[((size_t)e * NL + l) * MD + t] = thl[l];
  }
  if (abar) {
    double s = thl[0];
    for (int l = 1; l < NL; ++l) s += (double)(1 << l) * thl[l];
    abar[(size_t)e * MD + t] = s;
  }
}

// ---------------------------------------------------------------------------
// time step: max wave speed over all means (eq. euler-max-eigenvalue), FP64.
// Exact FP64 maximum in two passes: pass 1 estimates every mean's wave speed in
// FP32 from the high words of its FP64 values (20-bit mantissas, no FP64
// instruction) and keeps the FP32 maximum; means where the estimate is not
// reliable (a pressure below 1% of (gamma-1) E, values outside the FP32 range)
// are evaluated in FP64 at once. Pass 2 evaluates in FP64 only the means whose
// estimate is within 1% of the FP32 maximum. The estimate's relative error is
// below 2e-4 on reliable means, so the FP64 maximiser is among the candidates and
// the result is the same FP64 maximum as evaluating every mean.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float hi_f32(double x, bool& ok) {
  const int hi = __double2hiint(x);
  const int e = ((hi >> 20) & 0x7ff) - 896;   // exponent rebiased to FP32
  ok = ok && (e < 255);
  return __int_as_float(e > 0 ? ((hi & (int)0x80000000) | (e << 23) | ((hi & 0xfffff) << 3)) : (hi & (int)0x80000000));
}

template <int DIM, int MD>
__device__ __forceinline__ float lambda32(const double* q0, float g, bool& safe) {
  bool ok = true;
  const float r = hi_f32(q0[0], ok), E = hi_f32(q0[(DIM + 1) * MD], ok);
  const float inv = __frcp_rn(r);
  float kin = 0.f, vmax = 0.f;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const float m = hi_f32(q0[(1 + k) * MD], ok);
    const float vk = m * inv;
    kin = fmaf(m, vk, kin);
    vmax = fmaxf(vmax, fabsf(vk));
  }
  const float pr = (g - 1.f) * (E - 0.5f * kin);
  const float est = vmax + sqrtf(g * pr * inv);
  safe = ok && r > 0.f && E > 0.f && pr > 0.01f * (g - 1.f) * E && est <= 3.0e38f;
  return est;
}

template <int DIM, int MD>
__device__ __forceinline__ double lambda64(const double* q0, double gamma) {
  const double r = q0[0];
  const double inv = 1.0 / r;
  double kin = 0.0, vmax = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const double m = q0[(1 + k) * MD];
    kin = fma(m, m * inv, kin);
    vmax = fmax(vmax, fabs(m * inv));
  }
  const double pr = (gamma - 1.0) * (q0[(DIM + 1) * MD] - 0.5 * kin);
  return vmax + sqrt(gamma * pr * inv);
}

// block maxima: FP64 bits to lmax[0], FP32 bits to lmax[1] (non-negative values
// order like their bit patterns)
__device__ __forceinline__ void flush_lambda(double l64, float l32, bool bad, unsigned long long* lmax,
                                             long long* counters) {
  __shared__ double s64[32];
  __shared__ float s32[32];
  for (int o = 16; o > 0; o /= 2) {
    l64 = fmax(l64, __shfl_xor_sync(0xffffffffu, l64, o));
    l32 = fmaxf(l32, __shfl_xor_sync(0xffffffffu, l32, o));
  }
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  if (lane == 0) {
    s64[wid] = l64;
    s32[wid] = l32;
  }
  if (bad) atomicOr((unsigned long long*)&counters[0], 2ull);
  __syncthreads();
  if (threadIdx.x == 0) {
    double m64 = 0.0;
    float m32 = 0.f;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) {
      m64 = fmax(m64, s64[i]);
      m32 = fmaxf(m32, s32[i]);
    }
    if (m64 > 0.0) atomicMax(lmax, (unsigned long long)__double_as_longlong(m64));
    if (m32 > 0.f) atomicMax(lmax + 1, (unsigned long long)__float_as_uint(m32));
  }
  __syncthreads();
}

template <int DIM, int M>
__global__ void __launch_bounds__(256) k_lambda(KParams p, Work w, const double* __restrict__ u, int pass) {
  constexpr int MD = Geo<DIM, M>::MD, NV = Geo<DIM, M>::NV;
  const size_t n = (size_t)p.E * MD;
  const float g32 = (float)p.gamma;
  const float thr = (pass == 2) ? 0.99f * __uint_as_float((unsigned)w.lmax[1]) : 0.f;
  double l64 = 0.0;
  float l32 = 0.f;
  bool bad = false;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t e = i / MD, t = i % MD;
    const double* q0 = u + e * NV * MD + t;
    bool safe;
    const float est = lambda32<DIM, MD>(q0, g32, safe);
    const bool need = (pass == 1) ? !safe : (safe && est >= thr);
    if (pass == 1 && safe) l32 = fmaxf(l32, est);
    if (need) {
      const double lam = lambda64<DIM, MD>(q0, p.gamma);
      if (!isfinite(lam)) bad = true;
      else l64 = fmax(l64, lam);
    }
  }
  flush_lambda(l64, l32, bad, w.lmax, w.counters);
}

__global__ void k_dt(KParams p, Work w, double* dt_out) {
  const double lam = __longlong_as_double((long long)*w.lmax);
  const double denom = (double)(1 << (p.dim - 1)) * (2.0 * p.M - 1.0);
  const double dt = p.cfl * p.dxmin / (denom * lam);
  *w.dt = dt;
  if (dt_out) *dt_out = dt;
}

// ---------------------------------------------------------------------------
// batched persistent kernels: many problems of one (dim, M) in one launch; every
// CTA walks the concatenated element (or face-task) list with a grid stride and
// runs the single-problem body, so each problem sees exactly the standalone
// arithmetic
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_problem(const int* gstart, int nprob, int eg) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (gstart[mid] <= eg) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Resident CTAs per SM the batched K1 / K2 kernels must allow. Their per-problem
// parameters come from global memory instead of the kernel's constant bank, and
// without a bound the compiler keeps them in registers (up to twice the
// single-problem kernels' count, halving occupancy); these bounds cap the
// registers near the single-problem kernels' counts.
template <int DIM, int M>
struct K1BatchMinBlocks {
  static constexpr int v = sizeof(real) == 8 ? (DIM == 2 ? (M == 4 ? 21 : 12) : (M == 4 ? 10 : 1))
                                             : (DIM == 2 ? (M == 4 ? 32 : 16) : (M == 4 ? 16 : 2));
};
template <int DIM, int M>
struct K2BatchMinBlocks {
  static constexpr int v = sizeof(real) == 8 ? 4 : 5;
};

template <int DIM, int M>
__global__ void __launch_bounds__(Geo<DIM, M>::NT, K1BatchMinBlocks<DIM, M>::v)
    k_indicator_batch(BatchView b, const double* __restrict__ u) {
  extern __shared__ double sm[];
  for (int eg = blockIdx.x; eg < b.Etot; eg += gridDim.x) {
    const int k = find_problem(b.gstart, b.nprob, eg);
    indicator_body<DIM, M>(b.P[k], u + b.uoff[k], nullptr, b.W[k], eg - b.gstart[k], sm);
    __syncthreads();
  }
}

template <int DIM, int M>
__global__ void __launch_bounds__(128, K2BatchMinBlocks<DIM, M>::v) k_face_flux_batch(BatchView b) {
  for (int ti = blockIdx.x; ti < b.ntasks; ti += gridDim.x) {
    const FaceTask tk = b.ftasks[ti];
    face_body<DIM, M>(b.P[tk.prob], b.W[tk.prob], tk.dir, tk.nfaces, tk.first);
    __syncthreads();
  }
}

// mode 0: out = R(us); mode 1: out = ark u0 + brk (us + dt R(us)) with each
// problem's own dt from its workspace
template <int DIM, int M>
__global__ void __launch_bounds__(Geo<DIM, M>::NT, K3MinBlocks<DIM, M>::v)
    k_update_batch(BatchView b, const double* __restrict__ us, const double* __restrict__ u0, double* __restrict__ out,
                   double ark, double brk, int mode) {
  extern __shared__ double sm[];
  for (int eg = blockIdx.x; eg < b.Etot; eg += gridDim.x) {
    const int k = find_problem(b.gstart, b.nprob, eg);
    const Work& w = b.W[k];
    const long long o = b.uoff[k];
    update_body<DIM, M>(b.P[k], w, us + o, mode ? u0 + o : nullptr, out + o, ark, brk, 0.0, mode ? w.dt : nullptr,
                        mode, eg - b.gstart[k], sm, StageTerm{nullptr, 0.0, 1.0});
    __syncthreads();
  }
}

// Grid-wide barrier of a cooperative launch (every CTA resident): thread 0 of each
// CTA arrives on bar[0]; the last arrival resets it and advances the generation
// bar[1]; the others wait for the generation to change, at most `cap` polls
// (128 ns apart). Returns false (block-uniform) when this CTA gave up waiting.
__device__ __forceinline__ bool grid_sync(unsigned* bar, long long cap) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u) + 1u;
    if (arrived == gridDim.x) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long it = 0;
      while (*gen == g0) {
        if (++it > cap) {
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
  }
  return __syncthreads_or(ok) != 0 && __syncthreads_and(ok) != 0;
}

template <int DIM, int M>
struct FusedCfg {
  static constexpr int NT = Geo<DIM, M>::NT;
  static constexpr int NF = NT / Geo<DIM, M>::P;   // faces per face task (NF P = NT threads)
  static constexpr size_t a1 = K1Smem<DIM, M>::bytes, a3 = K3Smem<DIM, M>::bytes, a2 = FaceSmem<DIM, M, NF>::bytes;
  static constexpr size_t smem = (a1 > a3 ? (a1 > a2 ? a1 : a2) : (a3 > a2 ? a3 : a2));
  static constexpr int min_blocks = K1MinBlocks<DIM, M>::v < K3MinBlocks<DIM, M>::v ? K1MinBlocks<DIM, M>::v
                                                                                    : K3MinBlocks<DIM, M>::v;
};

// One RK stage of every problem of a group in one persistent launch: the indicator
// phase (K1) over all elements, a grid-wide barrier, the interface fluxes (K2) over
// all face tasks, a barrier, the update (K3) over all elements; each CTA walks the
// items with a grid stride, as the separate batched kernels do, so every problem
// sees the standalone arithmetic. A barrier that times out sets flag 4 of the first
// problem's status word and the kernel returns (the stage's output is then invalid).
template <int DIM, int M>
__global__ void __launch_bounds__(Geo<DIM, M>::NT, FusedCfg<DIM, M>::min_blocks)
    k_stage_fused(BatchView b, const double* __restrict__ us, const double* __restrict__ u0, double* __restrict__ out,
                  double ark, double brk, int mode, unsigned* bar, long long cap) {
  extern __shared__ double sm[];
  for (int eg = blockIdx.x; eg < b.Etot; eg += gridDim.x) {
    const int k = find_problem(b.gstart, b.nprob, eg);
    indicator_body<DIM, M>(b.P[k], us + b.uoff[k], nullptr, b.W[k], eg - b.gstart[k], sm);
    __syncthreads();
  }
  if (!grid_sync(bar, cap)) {
    if (threadIdx.x == 0) atomicOr((unsigned long long*)&b.W[0].counters[0], 4ull);
    return;
  }
  for (int ti = blockIdx.x; ti < b.ntasks_f; ti += gridDim.x) {
    const FaceTask tk = b.ftasks_f[ti];
    face_body_s<DIM, M, FusedCfg<DIM, M>::NF>(b.P[tk.prob], b.W[tk.prob], tk.dir, tk.nfaces, tk.first,
                                              reinterpret_cast<unsigned char*>(sm));
    __syncthreads();
  }
  if (!grid_sync(bar, cap)) {
    if (threadIdx.x == 0) atomicOr((unsigned long long*)&b.W[0].counters[0], 4ull);
    return;
  }
  for (int eg = blockIdx.x; eg < b.Etot; eg += gridDim.x) {
    const int k = find_problem(b.gstart, b.nprob, eg);
    const Work& w = b.W[k];
    const long long o = b.uoff[k];
    update_body<DIM, M>(b.P[k], w, us + o, mode ? u0 + o : nullptr, out + o, ark, brk, 0.0, mode ? w.dt : nullptr,
                        mode, eg - b.gstart[k], sm, StageTerm{nullptr, 0.0, 1.0});
    __syncthreads();
  }
}

// per-problem maximum wave speed, the two passes of k_lambda: each tile of
// kLambdaTile means lies in one problem; a CTA reduces its tile and flushes once
template <int DIM, int M>
__global__ void __launch_bounds__(256) k_lambda_batch(BatchView b, const double* __restrict__ u, int pass) {
  constexpr int MD = Geo<DIM, M>::MD, NV = Geo<DIM, M>::NV;
  for (int tile = blockIdx.x; tile < b.ltiles; tile += gridDim.x) {
    const int k = find_problem(b.lstart, b.nprob, tile);
    const KParams& p = b.P[k];
    const Work& w = b.W[k];
    const size_t n = (size_t)p.E * MD;
    const size_t i0 = (size_t)(tile - b.lstart[k]) * kLambdaTile;
    const size_t i1 = (i0 + kLambdaTile < n) ? i0 + kLambdaTile : n;
    const double* uk = u + b.uoff[k];
    const float g32 = (float)p.gamma;
    const float thr = (pass == 2) ? 0.99f * __uint_as_float((unsigned)w.lmax[1]) : 0.f;
    double l64 = 0.0;
    float l32 = 0.f;
    bool bad = false;
    for (size_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const size_t e = i / MD, t = i % MD;
      const double* q0 = uk + e * NV * MD + t;
      bool safe;
      const float est = lambda32<DIM, MD>(q0, g32, safe);
      const bool need = (pass == 1) ? !safe : (safe && est >= thr);
      if (pass == 1 && safe) l32 = fmaxf(l32, est);
      if (need) {
        const double lam = lambda64<DIM, MD>(q0, p.gamma);
        if (!isfinite(lam)) bad = true;
        else l64 = fmax(l64, lam);
      }
    }
    flush_lambda(l64, l32, bad, w.lmax, w.counters);
  }
}

__global__ void k_dt_batch(BatchView b) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= b.nprob) return;
  const KParams& p = b.P[k];
  const double lam = __longlong_as_double((long long)*b.W[k].lmax);
  const double denom = (double)(1 << (p.dim - 1)) * (2.0 * p.M - 1.0);
  *b.W[k].dt = p.cfl * p.dxmin / (denom * lam);
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
int upload_ops(int family) {
  DevOps ops;
  memset(&ops, 0, sizeof(ops));
  for (int l = 1; l <= 3; ++l) {
    LevelOps h;
    if (!make_level_ops(1 << l, family, &h)) return 1;
    DevLevel& d = ops.lv[l - 1];
    for (int i = 0; i < 64; ++i) {
      d.R[i] = (real)h.R[i];
      d.P[i] = (real)h.P[i];
      d.Dn[i] = (real)h.Dn[i];
      d.C[i] = (real)h.C[i];
    }
    for (int i = 0; i < 72; ++i) d.IRf[i] = (real)h.IRf[i];
    for (int i = 0; i < 8; ++i) {
      d.c0[i] = (real)h.c0[i];
      d.cn[i] = (real)h.cn[i];
      d.w[i] = (real)h.w[i];
    }
    const int n = 1 << l;
    double lr = 0.0, li = 0.0;
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += fabs(h.R[i * n + j]);
      lr = fmax(lr, s);
    }
    for (int k = 0; k <= n; ++k) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += fabs(h.IRf[k * n + j]);
      li = fmax(li, s);
    }
    d.lamR = (real)lr;
    d.lamI = (real)li;
  }
  cudaError_t err = cudaMemcpyToSymbol(c_ops, &ops, sizeof(DevOps), sizeof(DevOps) * family);
  if (err != cudaSuccess) return 2;
  DevLevelF opf[3];
  memset(opf, 0, sizeof(opf));
  for (int l = 1; l <= 3; ++l) {
    LevelOps h;
    if (!make_level_ops(1 << l, family, &h)) return 1;
    DevLevelF& d = opf[l - 1];
    for (int i = 0; i < 64; ++i) {
      d.R[i] = (float)h.R[i];
      d.Dn[i] = (float)h.Dn[i];
      d.Dna[i] = (float)fabs(h.Dn[i]);
    }
    for (int i = 0; i < 72; ++i) d.IRf[i] = (float)h.IRf[i];
    for (int i = 0; i < 8; ++i) d.w[i] = (float)h.w[i];
    const int n = 1 << l;
    double lr = 0.0, li = 0.0;
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += fabs((double)d.R[i * n + j]);
      lr = fmax(lr, s);
    }
    for (int k = 0; k <= n; ++k) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += fabs((double)d.IRf[k * n + j]);
      li = fmax(li, s);
    }
    d.lamR = (float)(lr * (1.0 + 1e-6));
    d.lamI = (float)(li * (1.0 + 1e-6));
  }
  err = cudaMemcpyToSymbol(c_opsf, opf, sizeof(opf), sizeof(opf) * family);
  return err == cudaSuccess ? 0 : 2;
}

namespace detail {

// Opt a kernel in to `bytes` of dynamic shared memory once per device (function
// attributes belong to a device's context); safe to call from several host threads.
template <typename K>
bool smem_attr_once(K* fn, size_t bytes, std::atomic<unsigned long long>& devices_done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
  const unsigned long long bit = 1ull << dev;
  if (devices_done.load(std::memory_order_acquire) & bit) return true;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) return false;
  devices_done.fetch_or(bit, std::memory_order_release);
  return true;
}

template <int DIM, int M>
int ind_impl(const KParams& p, const Work& w, const double* u, const double* frozen, cudaStream_t s) {
  constexpr size_t smem = K1Smem<DIM, M>::bytes;
  static std::atomic<unsigned long long> attr{0};
  if (!smem_attr_once(k_indicator<DIM, M>, smem, attr)) return 1;
  if (w.class_count && cudaMemsetAsync(w.class_count, 0, 16 * sizeof(int), s) != cudaSuccess) return 1;
  k_indicator<DIM, M><<<p.E, Geo<DIM, M>::NT, smem, s>>>(p, u, frozen, w);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <int DIM, int M>
int face_impl(const KParams& p, const Work& w, cudaStream_t s) {
  constexpr int NF = FaceCfg<DIM, M>::NF;
  for (int a = 0; a < DIM; ++a) {
    int nf = p.nfaces_along[a];
    for (int b = 0; b < DIM; ++b)
      if (b != a) nf *= p.nel[b];
    const int blocks = (nf + NF - 1) / NF;
    k_face_flux<DIM, M><<<blocks, 128, 0, s>>>(p, w, a, nf);
    if (cudaGetLastError() != cudaSuccess) return 1;
  }
  return 0;
}

template <int DIM, int M>
int upd_impl(const KParams& p, const Work& w, const double* us, const double* u0, double* out, double a, double b,
             double dt, const double* dt_dev, int mode, const StageTerm& x, cudaStream_t s) {
  constexpr size_t smem = K3Smem<DIM, M>::bytes;
  static std::atomic<unsigned long long> attr{0};
  if (!smem_attr_once(k_update<DIM, M>, smem, attr)) return 1;
  k_update<DIM, M><<<p.E, Geo<DIM, M>::NT, smem, s>>>(p, w, us, u0, out, a, b, dt, dt_dev, mode, x);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <int DIM, int M>
int pack_impl(const KParams& p, const Work& w, int a, int side, void* dst, cudaStream_t s) {
  int ntr = 1;
  for (int b = 0; b < DIM; ++b)
    if (b != a) ntr *= p.nel[b];
  const size_t n = (size_t)ntr * (Geo<DIM, M>::NV + Geo<DIM, M>::NL) * Geo<DIM, M>::P;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_pack_halo<DIM, M><<<blocks, 256, 0, s>>>(p, w, a, side, reinterpret_cast<real*>(dst), ntr);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <int DIM, int M>
int theta_impl(const KParams& p, const Work& w, double* theta, double* abar, cudaStream_t s) {
  k_theta<DIM, M><<<p.E, Geo<DIM, M>::NT, 0, s>>>(p, w, theta, abar);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <int DIM, int M>
int dt_impl(const KParams& p, const Work& w, const double* u, double* dt_out, cudaStream_t s) {
  if (cudaMemsetAsync(w.lmax, 0, 2 * sizeof(unsigned long long), s) != cudaSuccess) return 1;
  const size_t n = (size_t)p.E * Geo<DIM, M>::MD;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_lambda<DIM, M><<<blocks, 256, 0, s>>>(p, w, u, 1);
  k_lambda<DIM, M><<<blocks, 256, 0, s>>>(p, w, u, 2);
  k_dt<<<1, 1, 0, s>>>(p, w, dt_out);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace detail

namespace detail {

// dynamic shared-memory opt-in of the batched kernels, set once per device
// (the batch object calls batch_max_blocks at creation, before any capture)
template <int DIM, int M>
bool batch_attrs() {
  static std::atomic<unsigned long long> a1{0}, a3{0}, af{0};
  return smem_attr_once(k_indicator_batch<DIM, M>, K1Smem<DIM, M>::bytes, a1) &&
         smem_attr_once(k_update_batch<DIM, M>, K3Smem<DIM, M>::bytes, a3) &&
         smem_attr_once(k_stage_fused<DIM, M>, FusedCfg<DIM, M>::smem, af);
}

// one stage as one cooperative launch of k_stage_fused (grid: at most all CTAs resident)
template <int DIM, int M>
int bfused_impl(const BatchView& b, const double* us, const double* u0, double* out, double a, double bb, int mode,
                int grid, unsigned* bar, long long cap, cudaStream_t s) {
  if (!batch_attrs<DIM, M>()) return 1;
  if (cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s) != cudaSuccess) return 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(Geo<DIM, M>::NT);
  cfg.dynamicSmemBytes = FusedCfg<DIM, M>::smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_stage_fused<DIM, M>, b, us, u0, out, a, bb, mode, bar, cap) != cudaSuccess) return 1;
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <int DIM, int M>
int bind_impl(const BatchView& b, const double* u, int grid, cudaStream_t s) {
  if (!batch_attrs<DIM, M>()) return 1;
  k_indicator_batch<DIM, M><<<grid, Geo<DIM, M>::NT, K1Smem<DIM, M>::bytes, s>>>(b, u);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <int DIM, int M>
int bface_impl(const BatchView& b, int grid, cudaStream_t s) {
  k_face_flux_batch<DIM, M><<<grid, 128, 0, s>>>(b);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <int DIM, int M>
int bupd_impl(const BatchView& b, const double* us, const double* u0, double* out, double a, double bb, int mode,
              int grid, cudaStream_t s) {
  if (!batch_attrs<DIM, M>()) return 1;
  k_update_batch<DIM, M><<<grid, Geo<DIM, M>::NT, K3Smem<DIM, M>::bytes, s>>>(b, us, u0, out, a, bb, mode);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <int DIM, int M>
int bdt_impl(const BatchView& b, const double* u, int grid, cudaStream_t s) {
  k_lambda_batch<DIM, M><<<grid, 256, 0, s>>>(b, u, 1);
  k_lambda_batch<DIM, M><<<grid, 256, 0, s>>>(b, u, 2);
  k_dt_batch<<<(b.nprob + 127) / 128, 128, 0, s>>>(b);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// resident CTAs per SM of batched kernel `kind` (0 indicator, 1 face flux, 2 update, 3 wave speed,
// 4 the fused stage kernel)
template <int DIM, int M>
int bmax_impl(int kind) {
  if (!batch_attrs<DIM, M>()) return 0;
  int n = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (kind == 0)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_indicator_batch<DIM, M>, Geo<DIM, M>::NT,
                                                      K1Smem<DIM, M>::bytes);
  else if (kind == 1)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_face_flux_batch<DIM, M>, 128, 0);
  else if (kind == 2)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_update_batch<DIM, M>, Geo<DIM, M>::NT,
                                                      K3Smem<DIM, M>::bytes);
  else if (kind == 3)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_lambda_batch<DIM, M>, 256, 0);
  else if (kind == 4)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage_fused<DIM, M>, Geo<DIM, M>::NT,
                                                      FusedCfg<DIM, M>::smem);
  return e == cudaSuccess ? n : 0;
}

}  // namespace detail

#define SESC_BDISPATCH(FN, ...)                                              \
  do {                                                                       \
    if (dim == 2 && M == 4) return detail::FN<2, 4>(__VA_ARGS__);            \
    if (dim == 2 && M == 8) return detail::FN<2, 8>(__VA_ARGS__);            \
    if (dim == 3 && M == 4) return detail::FN<3, 4>(__VA_ARGS__);            \
    if (dim == 3 && M == 8) return detail::FN<3, 8>(__VA_ARGS__);            \
    return 1;                                                                \
  } while (0)

int launch_batch_indicator(const BatchView& b, int dim, int M, const double* u, int grid, void* stream) {
  SESC_BDISPATCH(bind_impl, b, u, grid, (cudaStream_t)stream);
}
int launch_batch_face_flux(const BatchView& b, int dim, int M, int grid, void* stream) {
  SESC_BDISPATCH(bface_impl, b, grid, (cudaStream_t)stream);
}
int launch_batch_update(const BatchView& b, int dim, int M, const double* us, const double* u0, double* out, double a,
                        double bb, int mode, int grid, void* stream) {
  SESC_BDISPATCH(bupd_impl, b, us, u0, out, a, bb, mode, grid, (cudaStream_t)stream);
}
int launch_batch_dt(const BatchView& b, int dim, int M, const double* u, int grid, void* stream) {
  SESC_BDISPATCH(bdt_impl, b, u, grid, (cudaStream_t)stream);
}
int launch_batch_stage_fused(const BatchView& b, int dim, int M, const double* us, const double* u0, double* out,
                             double a, double bb, int mode, int grid, unsigned* bar, long long cap, void* stream) {
  SESC_BDISPATCH(bfused_impl, b, us, u0, out, a, bb, mode, grid, bar, cap, (cudaStream_t)stream);
}
int fused_faces_per_task(int dim, int M) {
  if (dim == 2 && M == 4) return FusedCfg<2, 4>::NF;
  if (dim == 2 && M == 8) return FusedCfg<2, 8>::NF;
  if (dim == 3 && M == 4) return FusedCfg<3, 4>::NF;
  if (dim == 3 && M == 8) return FusedCfg<3, 8>::NF;
  return 0;
}
int batch_max_blocks(int dim, int M, int kind) {
  if (dim == 2 && M == 4) return detail::bmax_impl<2, 4>(kind);
  if (dim == 2 && M == 8) return detail::bmax_impl<2, 8>(kind);
  if (dim == 3 && M == 4) return detail::bmax_impl<3, 4>(kind);
  if (dim == 3 && M == 8) return detail::bmax_impl<3, 8>(kind);
  return 0;
}
#undef SESC_BDISPATCH

#define SESC_DISPATCH(FN, ...)                                      \
  do {                                                              \
    if (p.dim == 2 && p.M == 4) return detail::FN<2, 4>(__VA_ARGS__); \
    if (p.dim == 2 && p.M == 8) return detail::FN<2, 8>(__VA_ARGS__); \
    if (p.dim == 3 && p.M == 4) return detail::FN<3, 4>(__VA_ARGS__); \
    if (p.dim == 3 && p.M == 8) return detail::FN<3, 8>(__VA_ARGS__); \
    return 1;                                                       \
  } while (0)

int launch_indicator(const KParams& p, const Work& w, const double* u, const double* frozen, void* stream) {
  SESC_DISPATCH(ind_impl, p, w, u, frozen, (cudaStream_t)stream);
}
int launch_face_flux(const KParams& p, const Work& w, void* stream) {
  SESC_DISPATCH(face_impl, p, w, (cudaStream_t)stream);
}
int launch_update(const KParams& p, const Work& w, const double* us, const double* u0, double* out, double a,
                  double b, double dt, const double* dt_dev, int mode, void* stream) {
  const StageTerm x{nullptr, 0.0, 1.0};
  SESC_DISPATCH(upd_impl, p, w, us, u0, out, a, b, dt, dt_dev, mode, x, (cudaStream_t)stream);
}
int launch_update_x(const KParams& p, const Work& w, const double* us, const double* u0, double* out, double a,
                    double b, double dt, const double* dt_dev, const StageTerm& x, void* stream) {
  SESC_DISPATCH(upd_impl, p, w, us, u0, out, a, b, dt, dt_dev, 1, x, (cudaStream_t)stream);
}
int launch_pack_halo(const KParams& p, const Work& w, int a, int side, void* dst, void* stream) {
  SESC_DISPATCH(pack_impl, p, w, a, side, dst, (cudaStream_t)stream);
}
int launch_theta(const KParams& p, const Work& w, double* theta, double* abar, void* stream) {
  SESC_DISPATCH(theta_impl, p, w, theta, abar, (cudaStream_t)stream);
}
int launch_dt(const KParams& p, const Work& w, const double* u, double* dt_out, void* stream) {
  SESC_DISPATCH(dt_impl, p, w, u, dt_out, (cudaStream_t)stream);
}

#undef SESC_DISPATCH

}  // namespace SESC_NS
}  // namespace sesc
