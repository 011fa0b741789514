// FP64 kernels of the multi-level blended DG/FV right-hand side.
//
// Kernels (one CTA per element for K1/K3, a group of faces per CTA for K2):
//   K1 k_indicator  reconstruction per level, positivity squeezing (eq. calc-
//                   squeezing-parameter, two-step reading), smoothness sigma and
//                   blending factor (eqs. L1-norm-slope, calc-blending-factor), the
//                   high-to-low snapping loop of the multi-level sketch, blending
//                   weights (eq. blending-weights) and the blended face-centred
//                   states of the 2d element faces (eq. 3D-prolongation generalised
//                   to all levels).
//   K2 k_face_flux  blended common interface flux at element faces: FV candidate
//                   f*(Ubar_L, Ubar_R) and level-n candidates P f*(R Ubar R^T) P^T
//                   (eqs. 3D-boundary-value-recon ... 3D-blend-interface-fluxes),
//                   weights (theta_L + theta_R)/2.
//   K3 k_update     inner subcell interface fluxes, level right-hand sides
//                   (eq. multilevel-blending-scheme in the n-mode form of
//                   eq. dgfv-scheme-3d), their theta blend, and the RK stage.
//   k_lambda/k_dt   time step of eq. cfl-condition.
// Layouts: see include/sesc.h. Everything here is FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "kparams.h"
#include "opgen.h"

namespace sesc {

// ---------------------------------------------------------------------------
// operator tables in constant memory: [family][M == 8][log2 n]
// ---------------------------------------------------------------------------
struct DevLevel {
  double R[64], P[64], Dn[64], Dhat[64], IRf[72], Bh0[8], Bhn[8], w[8];
};
struct DevOps {
  DevLevel lv[4];
};
__constant__ DevOps c_ops[2];

// ---------------------------------------------------------------------------
// compile-time geometry
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int ipow(int b, int e) { return e == 0 ? 1 : b * ipow(b, e - 1); }
__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n / 2); }
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
  static constexpr int FAM = 0;
};

__device__ __forceinline__ const DevLevel& lev(int family, int l) { return c_ops[family].lv[l]; }

// ---------------------------------------------------------------------------
// Euler physics (eqs. comp-euler-conservative, equation-of-state) and HLL with
// Einfeldt speeds: Roe averages, S_L = min(v_L - c_L, v^ - c^),
// S_R = max(v_R + c_R, v^ + c^); sound speeds sqrt(max(gamma p / rho, 0)) so that
// a squeezed state whose pressure (target 1e-20) rounds below zero gives 0.
// ---------------------------------------------------------------------------
template <int DIM>
__device__ __forceinline__ double pressure(const double* q, double g) {
  double kin = q[1] * q[1];
#pragma unroll
  for (int k = 1; k < DIM; ++k) kin += q[1 + k] * q[1 + k];
  kin = kin / q[0];
  return (g - 1.0) * (q[DIM + 1] - 0.5 * kin);
}

template <int DIM>
__device__ __forceinline__ bool permissible(const double* q, double g) {
  return q[0] > 0.0 && pressure<DIM>(q, g) > 0.0;
}

// primitive view of a conserved state with one reciprocal of the density
template <int DIM>
struct Prim {
  double rho, inv, v[DIM], p;
  __device__ __forceinline__ void load(const double* q, double g) {
    rho = q[0];
    inv = 1.0 / rho;
    double kin = 0.0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      v[k] = q[1 + k] * inv;
      kin = fma(q[1 + k], v[k], kin);
    }
    p = (g - 1.0) * (q[DIM + 1] - 0.5 * kin);
  }
};

// Euler flux in direction a from the conserved state and its primitive view
template <int DIM>
__device__ __forceinline__ void flux_of(const double* q, const Prim<DIM>& w, int a, double* f) {
  const double va = w.v[a];
  f[0] = q[1 + a];
#pragma unroll
  for (int k = 0; k < DIM; ++k) f[1 + k] = q[1 + k] * va;
  f[1 + a] += w.p;
  f[DIM + 1] = va * (q[DIM + 1] + w.p);
}

template <int DIM>
__device__ void hll(const double* uL, const double* uR, int a, double g, double* F) {
  constexpr int NV = DIM + 2;
  Prim<DIM> L, R;
  L.load(uL, g);
  R.load(uR, g);
  const double cL = sqrt(fmax(g * L.p * L.inv, 0.0)), cR = sqrt(fmax(g * R.p * R.inv, 0.0));
  const double HL = (uL[NV - 1] + L.p) * L.inv, HR = (uR[NV - 1] + R.p) * R.inv;
  const double sL = sqrt(L.rho), sR = sqrt(R.rho);
  const double is = 1.0 / (sL + sR);
  double vh[DIM], v2 = 0.0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    vh[k] = (sL * L.v[k] + sR * R.v[k]) * is;
    v2 = fma(vh[k], vh[k], v2);
  }
  const double Hh = (sL * HL + sR * HR) * is;
  const double c2 = (g - 1.0) * (Hh - 0.5 * v2);
  const double ch = sqrt(fmax(c2, 0.0));
  const double SL = fmin(L.v[a] - cL, vh[a] - ch);
  const double SR = fmax(R.v[a] + cR, vh[a] + ch);
  if (SL >= 0.0) {
    flux_of<DIM>(uL, L, a, F);
    return;
  }
  if (SR <= 0.0) {
    flux_of<DIM>(uR, R, a, F);
    return;
  }
  double fL[NV], fR[NV];
  flux_of<DIM>(uL, L, a, fL);
  flux_of<DIM>(uR, R, a, fR);
  const double inv = 1.0 / (SR - SL);
  const double sls = SL * SR;
#pragma unroll
  for (int v = 0; v < NV; ++v) F[v] = (SR * fL[v] - SL * fR[v] + sls * (uR[v] - uL[v])) * inv;
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
template <int M>
__device__ __forceinline__ int stride_of(int a) { return a == 0 ? 1 : (a == 1 ? M : M * M); }

// sub-element index of subcell t at level n (x fastest), and local index within it
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

// segmented tree reduction over contiguous segments of SZ entries of NVV rows of
// length MD; result at position s*SZ of each row. Includes the barriers.
template <int MD, int NVV, bool MIN>
__device__ void seg_reduce(double* red, int SZ, int t) {
  for (int st = SZ / 2; st >= 1; st /= 2) {
    __syncthreads();
    if (t < MD && (t % SZ) < st) {
#pragma unroll
      for (int v = 0; v < NVV; ++v) {
        const double x = red[v * MD + t], y = red[v * MD + t + st];
        red[v * MD + t] = MIN ? fmin(x, y) : (x + y);
      }
    }
  }
  __syncthreads();
}

// blockwise n-mode product along axis a: out[v][t] = sum_j A[i][j] in[v][t + (j - i) stride]
template <int DIM, int M, int N, int NVV>
__device__ __forceinline__ void mode_sq(double* out, const double* in, const double* A, int a, int t) {
  constexpr int MD = ipow(M, DIM);
  if (t >= MD) return;
  const int st = stride_of<M>(a);
  const int c = (a == 0) ? (t % M) : (a == 1 ? (t / M) % M : t / (M * M));
  const int i = c % N;
  const int base = t - i * st;
#pragma unroll
  for (int v = 0; v < NVV; ++v) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < N; ++j) s = fma(A[i * N + j], in[v * MD + base + j * st], s);
    out[v * MD + t] = s;
  }
}

// reconstruction of the level-N polynomial of every sub-element: ut = u x_0 R x_1 R (x_2 R)
template <int DIM, int M, int N>
__device__ void reconstruct(double* ut, double* tmp, const double* su, int family, int t) {
  constexpr int NV = DIM + 2;
  const double* R = lev(family, ilog2(N)).R;
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

// value of the level-n polynomial of subcell t's sub-element at one interface along a:
// row = interface index within the sub-element (0..n); from the n means via IRf.
template <int DIM, int M, int N>
__device__ __forceinline__ void interface_value(const double* su, int t, int a, int row, int family, double* U) {
  constexpr int MD = ipow(M, DIM);
  constexpr int NV = DIM + 2;
  const double* IRf = lev(family, ilog2(N)).IRf;
  const int st = stride_of<M>(a);
  const int c = (a == 0) ? (t % M) : (a == 1 ? (t / M) % M : t / (M * M));
  const int first = t - (c % N) * st;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    double s = 0.0;
#pragma unroll
    for (int j = 0; j < N; ++j) s = fma(IRf[row * N + j], su[v * MD + first + j * st], s);
    U[v] = s;
  }
}

// density only of interface_value (first step of the squeezing)
template <int DIM, int M, int N>
__device__ __forceinline__ double interface_density(const double* su, int t, int a, int row, int family) {
  const double* IRf = lev(family, ilog2(N)).IRf;
  const int st = stride_of<M>(a);
  const int c = (a == 0) ? (t % M) : (a == 1 ? (t / M) % M : t / (M * M));
  const int first = t - (c % N) * st;
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < N; ++j) s = fma(IRf[row * N + j], su[first + j * st], s);
  return s;
}

// blended state at the right (side = 1) or left (side = 0) face of subcell t along a:
// theta^(1) u_t + sum_n theta^(n) ((1 - beta) <u> + beta U^(n)) (reading R1).
template <int DIM, int M>
__device__ void blended_face_state(const double* su, const double* thtab, const double* beta_s,
                                   const double* avg_s, int t, int a, int side, int family, double* Ub) {
  constexpr int MD = ipow(M, DIM);
  constexpr int NV = DIM + 2;
  constexpr int NL = ilog2(M) + 1;
  const double th1 = thtab[t];
#pragma unroll
  for (int v = 0; v < NV; ++v) Ub[v] = (th1 != 0.0) ? th1 * su[v * MD + t] : 0.0;
  const int c = (a == 0) ? (t % M) : (a == 1 ? (t / M) % M : t / (M * M));
#pragma unroll
  for (int l = 1; l < NL; ++l) {
    const double th = thtab[l * MD + t];
    if (th == 0.0) continue;
    const int n = 1 << l;
    const int row = (c % n) + side;
    double U[NV];
    if (n == 2) interface_value<DIM, M, 2>(su, t, a, row, family, U);
    else if (n == 4) interface_value<DIM, M, 4>(su, t, a, row, family, U);
    else interface_value<DIM, M, (M >= 8 ? 8 : 4)>(su, t, a, row, family, U);
    const int s = sub_index<DIM, M>(t, n);
    const int off = s_off(M, DIM, n);
    const double b = beta_s[off + s];
    if (b != 1.0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) U[v] = (1.0 - b) * avg_s[v * Geo<DIM, M>::S + off + s] + b * U[v];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) Ub[v] += th * U[v];
  }
}

// ---------------------------------------------------------------------------
// Blended common flux on a group of NF faces with P transverse points each
// (readings R2 / R7). Thread tid < NF*P handles face f = tid / P, point j = tid % P.
// Scratch: sUL, sUR, sT, sF each NF*NV*P doubles, sflag NF*P ints.
// ---------------------------------------------------------------------------
template <int DIM, int M, int N>
__device__ __forceinline__ void transverse(const double* src, double* sT, const double* A, int f, int j,
                                           bool valid, double* out) {
  constexpr int NV = DIM + 2;
  constexpr int P = ipow(M, DIM - 1);
  if (DIM == 2) {
    if (valid) {
      const int i = j % N, base = j - i;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        double s = 0.0;
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
        double s = 0.0;
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
        double s = 0.0;
#pragma unroll
        for (int k = 0; k < N; ++k) s = fma(A[i1 * N + k], sT[(f * NV + v) * P + b1 + k * M], s);
        out[v] = s;
      }
    }
    __syncthreads();
  }
}

template <int DIM, int M, int N>
__device__ void level_candidate(const double* UL, const double* UR, double wl, int a, double g, int family,
                                int f, int j, bool valid, double* sUL, double* sUR, double* sT, double* sF,
                                int* sflag, bool& have1, double* F1, double* Fout, long long* counters) {
  constexpr int NV = DIM + 2;
  constexpr int P = ipow(M, DIM - 1);
  const DevLevel& L = lev(family, ilog2(N));
  double rL[NV], rR[NV];
  transverse<DIM, M, N>(sUL, sT, L.R, f, j, valid, rL);
  transverse<DIM, M, N>(sUR, sT, L.R, f, j, valid, rR);
  const bool ok = valid && permissible<DIM>(rL, g) && permissible<DIM>(rR, g);
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
  double Fn[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Fn[v] = 0.0;
  if (blk) hll<DIM>(rL, rR, a, g, Fn);
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) sF[(f * NV + v) * P + j] = Fn[v];
  }
  __syncthreads();
  double Fp[NV];
  transverse<DIM, M, N>(sF, sT, L.P, f, j, valid, Fp);
  if (valid && wl != 0.0) {
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
      bool first = (DIM == 2) ? (j % N == 0) : ((j % M) % N == 0 && ((j / M) % N) == 0);
      if (first) atomicAdd((unsigned long long*)&counters[2], 1ull);
    }
  }
  __syncthreads();
}

template <int DIM, int M>
__device__ void blended_flux(const double* UL, const double* UR, const double* w, int a, double g, int family,
                             int f, int j, bool valid, double* sUL, double* sUR, double* sT, double* sF,
                             int* sflag, double* Fout, long long* counters) {
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
  double F1[NV];
  bool have1 = false;
#pragma unroll
  for (int v = 0; v < NV; ++v) Fout[v] = 0.0;
  if (valid && w[0] != 0.0) {
    hll<DIM>(UL, UR, a, g, F1);
    have1 = true;
#pragma unroll
    for (int v = 0; v < NV; ++v) Fout[v] = w[0] * F1[v];
  }
  __syncthreads();
#pragma unroll
  for (int l = 1; l < NL; ++l) {
    if (!__syncthreads_or(valid && w[l] != 0.0)) continue;
    if (l == 1) level_candidate<DIM, M, 2>(UL, UR, w[l], a, g, family, f, j, valid, sUL, sUR, sT, sF, sflag, have1, F1, Fout, counters);
    else if (l == 2) level_candidate<DIM, M, 4>(UL, UR, w[l], a, g, family, f, j, valid, sUL, sUR, sT, sF, sflag, have1, F1, Fout, counters);
    else level_candidate<DIM, M, (M >= 8 ? 8 : 4)>(UL, UR, w[l], a, g, family, f, j, valid, sUL, sUR, sT, sF, sflag, have1, F1, Fout, counters);
  }
}

// ---------------------------------------------------------------------------
// K1: indicator, coefficients, blending weights and element face states
// ---------------------------------------------------------------------------
template <int DIM, int M>
struct K1Smem {
  static constexpr int MD = Geo<DIM, M>::MD, NV = Geo<DIM, M>::NV, S = Geo<DIM, M>::S, NL = Geo<DIM, M>::NL;
  // doubles
  static constexpr int o_su = 0;
  static constexpr int o_ut = o_su + NV * MD;
  static constexpr int o_tmp = o_ut + NV * MD;
  static constexpr int o_red = o_tmp + NV * MD;
  static constexpr int o_th = o_red + NV * MD;
  static constexpr int o_avg = o_th + NL * MD;
  static constexpr int o_sig = o_avg + NV * S;
  static constexpr int o_alpha = o_sig + NV * S;
  static constexpr int o_beta = o_alpha + S;
  static constexpr int o_brho = o_beta + S;
  static constexpr int total = o_brho + S;
  static constexpr size_t bytes = sizeof(double) * total;
};

// per-sub-element averages of level N into avg[v][off + s]
template <int DIM, int M, int N>
__device__ void sub_averages(const double* su, double* red, double* avg, int t) {
  constexpr int MD = ipow(M, DIM), NV = DIM + 2, S = Geo<DIM, M>::S;
  constexpr int SZ = ipow(N, DIM);
  constexpr int NS = ipow(M / N, DIM);
  constexpr int off = s_off(M, DIM, N);
  __syncthreads();
  if (t < MD) {
    const int pos = seg_pos<DIM, M>(t, N);
#pragma unroll
    for (int v = 0; v < NV; ++v) red[v * MD + pos] = su[v * MD + t];
  }
  seg_reduce<MD, NV, false>(red, SZ, t);
  if (t < NS * NV) {
    const int v = t / NS, s = t % NS;
    avg[v * S + off + s] = red[v * MD + s * SZ] / (double)SZ;
  }
  __syncthreads();
}

// sigma^(N) per primitive variable and sub-element (reading R3), from ut (unlimited nodal)
template <int DIM, int M, int N>
__device__ void smoothness(const double* ut, double* tmp, double* red, double* sig, double g, int family, int t) {
  constexpr int MD = ipow(M, DIM), NV = DIM + 2, S = Geo<DIM, M>::S;
  constexpr int SZ = ipow(N, DIM);
  constexpr int NS = ipow(M / N, DIM);
  constexpr int off = s_off(M, DIM, N);
  const DevLevel& L = lev(family, ilog2(N));
  // primitives at the nodes
  if (t < MD) {
    double q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = ut[v * MD + t];
    tmp[t] = q[0];
#pragma unroll
    for (int k = 0; k < DIM; ++k) tmp[(1 + k) * MD + t] = q[1 + k] / q[0];
    tmp[(NV - 1) * MD + t] = pressure<DIM>(q, g);
  }
  __syncthreads();
  if (t < MD) {
    double W = L.w[(t % M) % N] * L.w[((t / M) % M) % N];
    if (DIM == 3) W *= L.w[(t / (M * M)) % N];
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int st = stride_of<M>(a);
      const int c = (a == 0) ? (t % M) : (a == 1 ? (t / M) % M : t / (M * M));
      const int i = c % N, base = t - i * st;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        double s = 0.0;
#pragma unroll
        for (int j = 0; j < N; ++j) s = fma(L.Dn[i * N + j], tmp[v * MD + base + j * st], s);
        acc[v] += fabs(s) * W;
      }
    }
    const int pos = seg_pos<DIM, M>(t, N);
#pragma unroll
    for (int v = 0; v < NV; ++v) red[v * MD + pos] = acc[v];
  }
  seg_reduce<MD, NV, false>(red, SZ, t);
  if (t < NS * NV) {
    const int v = t / NS, s = t % NS;
    const double h = (double)N / (double)M;
    const double hd = (DIM == 2) ? h : h * h;
    sig[v * S + off + s] = hd * red[v * MD + s * SZ];
  }
  __syncthreads();
}

// squeezing parameter beta^(N) per sub-element (reading R4, two steps)
template <int DIM, int M, int N>
__device__ void squeeze(const double* su, const double* ut, double* red, const double* avg, double* beta,
                        double* brho, double g, int family, int t, long long* counters) {
  constexpr int MD = ipow(M, DIM), NV = DIM + 2, S = Geo<DIM, M>::S;
  constexpr int SZ = ipow(N, DIM);
  constexpr int NS = ipow(M / N, DIM);
  constexpr int off = s_off(M, DIM, N);
  const int s = (t < MD) ? sub_index<DIM, M>(t, N) : 0;
  const int pos = (t < MD) ? seg_pos<DIM, M>(t, N) : 0;
  // step 1: density minimum over nodes and owned face points
  if (t < MD) {
    double rmin = ut[t];
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int c = (a == 0) ? (t % M) : (a == 1 ? (t / M) % M : t / (M * M));
      const int i = c % N;
      rmin = fmin(rmin, interface_density<DIM, M, N>(su, t, a, i, family));
      if (i == N - 1) rmin = fmin(rmin, interface_density<DIM, M, N>(su, t, a, N, family));
    }
    red[pos] = rmin;
  }
  seg_reduce<MD, 1, true>(red, SZ, t);
  if (t < NS) {
    double q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = avg[v * S + off + t];
    const double ravg = q[0], pavg = pressure<DIM>(q, g);
    const double eps = fmin(fmin(1e-20, ravg), pavg);
    const double rmin = red[t * SZ];
    double b = (rmin >= eps) ? 1.0 : (ravg - eps) / (ravg - rmin);
    brho[off + t] = fmin(b, 1.0);
  }
  __syncthreads();
  // step 2: pressure minimum over the density-squeezed points
  if (t < MD) {
    const double br = brho[off + s];
    double av[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) av[v] = avg[v * S + off + s];
    double q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = (br == 1.0) ? ut[v * MD + t] : (1.0 - br) * av[v] + br * ut[v * MD + t];
    double pmin = pressure<DIM>(q, g);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int c = (a == 0) ? (t % M) : (a == 1 ? (t / M) % M : t / (M * M));
      const int i = c % N;
      for (int side = 0; side < 2; ++side) {
        if (side == 1 && i != N - 1) break;
        double U[NV];
        interface_value<DIM, M, N>(su, t, a, i + side, family, U);
        if (br != 1.0) {
#pragma unroll
          for (int v = 0; v < NV; ++v) U[v] = (1.0 - br) * av[v] + br * U[v];
        }
        pmin = fmin(pmin, pressure<DIM>(U, g));
      }
    }
    red[pos] = pmin;
  }
  seg_reduce<MD, 1, true>(red, SZ, t);
  if (t < NS) {
    double q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = avg[v * S + off + t];
    const double ravg = q[0], pavg = pressure<DIM>(q, g);
    const double eps = fmin(fmin(1e-20, ravg), pavg);
    const double pmin = red[t * SZ];
    double bp = (pmin >= eps) ? 1.0 : (pavg - eps) / (pavg - pmin);
    bp = fmin(bp, 1.0);
    double b = brho[off + t] * bp;
    if (!(ravg > 0.0 && pavg > 0.0) || !isfinite(b)) b = 0.0;
    b = fmax(b, 0.0);
    beta[off + t] = b;
    if (b < 1.0) atomicAdd((unsigned long long*)&counters[1], 1ull);
  }
  __syncthreads();
}

// raw blending factor of level NP (= 2 N) from sigma^(NP), the children sums of
// sigma^(N) and beta^(NP), written to alpha[]. eq. calc-blending-factor.
template <int DIM, int M, int NP>
__device__ void blending_factor(const double* sig, const double* beta, double* alpha, double tauA, double tauS,
                                double betaL, int t) {
  constexpr int NV = DIM + 2, S = Geo<DIM, M>::S;
  constexpr int NSP = ipow(M / NP, DIM);
  constexpr int kp = M / NP, kc = M / (NP / 2);
  constexpr int offp = s_off(M, DIM, NP), offc = s_off(M, DIM, NP / 2);
  if (t < NSP) {
    const int px = t % kp, py = (t / kp) % kp, pz = (DIM == 3) ? t / (kp * kp) : 0;
    double amin = 1.0;
    bool first = true;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      // children sum: pairs along x, then y, then z
      double cs;
      {
        double yz[2][2];
        for (int dz = 0; dz < (DIM == 3 ? 2 : 1); ++dz)
          for (int dy = 0; dy < 2; ++dy) {
            const int cx = 2 * px, cy = 2 * py + dy, cz = 2 * pz + dz;
            const int c0 = cx + kc * (cy + kc * cz);
            yz[dz][dy] = sig[v * S + offc + c0] + sig[v * S + offc + c0 + 1];
          }
        cs = yz[0][0] + yz[0][1];
        if (DIM == 3) cs = cs + (yz[1][0] + yz[1][1]);
      }
      const double sp = sig[v * S + offp + t];
      double av;
      const bool fin = isfinite(sp) && isfinite(cs);
      const double ratio = fabs(sp - cs) / fmax(fmax(sp, cs), 1.0);
      if (!fin || !isfinite(ratio)) av = 0.0;
      else av = 1.0 - fmin(fmax(tauA * (ratio - tauS), 0.0), 1.0);
      amin = first ? av : fmin(amin, av);
      first = false;
    }
    if (beta[offp + t] < betaL) amin = 0.0;
    alpha[offp + t] = amin;
  }
  __syncthreads();
}

// snap level n; returns true if all sub-elements exceeded alpha_H (loop ends)
template <int DIM, int M, int N>
__device__ bool snap(double* alpha, double alphaH, double alphaL, int t) {
  constexpr int NS = ipow(M / N, DIM);
  constexpr int off = s_off(M, DIM, N);
  const double a = (t < NS) ? alpha[off + t] : 0.0;
  const bool all_hi = __syncthreads_and(t < NS ? (a > alphaH) : true);
  const bool all_lo = __syncthreads_and(t < NS ? (a < alphaL) : true);
  if (t < NS) {
    if (all_hi) alpha[off + t] = 1.0;
    else if (all_lo) alpha[off + t] = 0.0;
  }
  __syncthreads();
  return all_hi;
}

template <int DIM, int M, int N>
__device__ void level_stats(const double* su, double* ut, double* tmp, double* red, double* avg, double* sig,
                            double g, int family, int t) {
  sub_averages<DIM, M, N>(su, red, avg, t);
  reconstruct<DIM, M, N>(ut, tmp, su, family, t);
  smoothness<DIM, M, N>(ut, tmp, red, sig, g, family, t);
}

template <int DIM, int M>
__global__ void __launch_bounds__(Geo<DIM, M>::NT) k_indicator(KParams p, const double* __restrict__ u,
                                                               const double* __restrict__ frozen, Work w) {
  constexpr int MD = Geo<DIM, M>::MD, NV = Geo<DIM, M>::NV, S = Geo<DIM, M>::S, NL = Geo<DIM, M>::NL;
  constexpr int P = Geo<DIM, M>::P, NT = Geo<DIM, M>::NT;
  using L = K1Smem<DIM, M>;
  extern __shared__ double sm[];
  double* su = sm + L::o_su;
  double* ut = sm + L::o_ut;
  double* tmp = sm + L::o_tmp;
  double* red = sm + L::o_red;
  double* th = sm + L::o_th;
  double* avg = sm + L::o_avg;
  double* sig = sm + L::o_sig;
  double* alpha = sm + L::o_alpha;
  double* beta = sm + L::o_beta;
  double* brho = sm + L::o_brho;
  const int t = threadIdx.x;
  const int e = blockIdx.x;
  const double g = p.gamma;
  const int fam = p.family;
  const double* ue = u + (size_t)e * NV * MD;
  for (int i = t; i < NV * MD; i += NT) su[i] = ue[i];
  for (int i = t; i < S; i += NT) { alpha[i] = 0.0; beta[i] = 1.0; }
  __syncthreads();
  // non-permissible mean values (rho <= 0 or 2 rho E <= |m|^2)
  if (t < MD) {
    const double r = su[t];
    double m2 = 0.0;
#pragma unroll
    for (int k = 0; k < DIM; ++k) m2 += su[(1 + k) * MD + t] * su[(1 + k) * MD + t];
    if (!(r > 0.0) || !(2.0 * r * su[(NV - 1) * MD + t] > m2)) atomicOr((unsigned long long*)&w.counters[0], 1ull);
  }
  if (frozen != nullptr) {
    const double* fe = frozen + (size_t)e * 2 * S;
    for (int i = t; i < S; i += NT) { alpha[i] = fe[i]; beta[i] = fe[S + i]; }
    sub_averages<DIM, M, 2>(su, red, avg, t);
    sub_averages<DIM, M, 4>(su, red, avg, t);
    if (M == 8) sub_averages<DIM, M, (M >= 8 ? 8 : 4)>(su, red, avg, t);
  } else {
    // top level
    level_stats<DIM, M, M>(su, ut, tmp, red, avg, sig, g, fam, t);
    squeeze<DIM, M, M>(su, ut, red, avg, beta, brho, g, fam, t, w.counters);
    bool stopped = false;
    if (M == 8) {
      level_stats<DIM, M, 4>(su, ut, tmp, red, avg, sig, g, fam, t);
      blending_factor<DIM, M, (M >= 8 ? 8 : 4)>(sig, beta, alpha, p.tauA, p.tauS, p.betaL, t);
      stopped = snap<DIM, M, (M >= 8 ? 8 : 4)>(alpha, p.alphaH, p.alphaL, t);
      if (!stopped) squeeze<DIM, M, 4>(su, ut, red, avg, beta, brho, g, fam, t, w.counters);
    }
    if (!stopped) {
      level_stats<DIM, M, 2>(su, ut, tmp, red, avg, sig, g, fam, t);
      blending_factor<DIM, M, 4>(sig, beta, alpha, p.tauA, p.tauS, p.betaL, t);
      stopped = snap<DIM, M, 4>(alpha, p.alphaH, p.alphaL, t);
      if (!stopped) {
        squeeze<DIM, M, 2>(su, ut, red, avg, beta, brho, g, fam, t, w.counters);
        constexpr int NS2 = ipow(M / 2, DIM);
        constexpr int off2 = s_off(M, DIM, 2);
        if (t < NS2) {
          const double b = beta[off2 + t];
          alpha[off2 + t] = (b < p.betaL) ? 0.0 : b;   // alpha^(2) := beta^(2)
        }
        __syncthreads();
        snap<DIM, M, 2>(alpha, p.alphaH, p.alphaL, t);
      }
    }
  }
  __syncthreads();
  // blending weights per subcell (eq. blending-weights)
  if (t < MD) {
    double rest = 1.0;
#pragma unroll
    for (int l = NL - 1; l >= 1; --l) {
      const int n = 1 << l;
      const double A = alpha[s_off(M, DIM, n) + sub_index<DIM, M>(t, n)];
      th[l * MD + t] = A * rest;
      rest = rest * (1.0 - A);
    }
    th[t] = rest;
  }
  __syncthreads();
  // level bounds of the element
  int used = 0;
#pragma unroll
  for (int l = 0; l < NL; ++l) used |= __syncthreads_or(t < MD && th[l * MD + t] != 0.0) ? (1 << l) : 0;
  if (t == 0) {
    int lo = 0, hi = 0;
    for (int l = 0; l < NL; ++l)
      if (used & (1 << l)) { lo = l; break; }
    for (int l = NL - 1; l >= 0; --l)
      if (used & (1 << l)) { hi = l; break; }
    w.decision[e] = (uint8_t)(lo | (hi << 4));
    atomicAdd((unsigned long long*)&w.counters[4 + lo], 1ull);
    atomicAdd((unsigned long long*)&w.counters[8 + hi], 1ull);
  }
  // coefficients out
  double* ce = w.coeffs + (size_t)e * 2 * S;
  for (int i = t; i < S; i += NT) { ce[i] = alpha[i]; ce[S + i] = beta[i]; }
  // blended states of the element faces and their weights
  for (int i = t; i < 2 * DIM * P; i += NT) {
    const int face = i / P, j = i % P, a = face / 2, side = face % 2;
    const int ca = side ? M - 1 : 0;
    int coords[3];
    coords[a] = ca;
    if (DIM == 2) {
      coords[1 - a] = j;
    } else {
      const int b0 = (a == 0) ? 1 : 0, b1 = (a == 2) ? 1 : 2;
      coords[b0] = j % M;
      coords[b1] = j / M;
    }
    int tt = coords[0] + M * coords[1];
    if (DIM == 3) tt += M * M * coords[2];
    double Ub[NV];
    blended_face_state<DIM, M>(su, th, beta, avg, tt, a, side, fam, Ub);
    double* fs = w.face_states + ((size_t)e * 2 * DIM + face) * (NV + NL) * P;
#pragma unroll
    for (int v = 0; v < NV; ++v) fs[v * P + j] = Ub[v];
#pragma unroll
    for (int l = 0; l < NL; ++l) fs[(NV + l) * P + j] = th[l * MD + tt];
  }
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

template <int DIM, int M>
__global__ void __launch_bounds__(128) k_face_flux(KParams p, Work w, int a, int nfaces) {
  constexpr int NV = Geo<DIM, M>::NV, NL = Geo<DIM, M>::NL, P = Geo<DIM, M>::P;
  constexpr int NF = FaceCfg<DIM, M>::NF;
  __shared__ double sUL[NF * NV * P], sUR[NF * NV * P], sT[NF * NV * P], sF[NF * NV * P];
  __shared__ int sflag[NF * P];
  const int tid = threadIdx.x;
  const int f = tid / P, j = tid % P;
  const int fid = blockIdx.x * NF + f;
  const bool valid = fid < nfaces;
  double UL[NV], UR[NV], wl[NL];
  if (valid) {
    const int NA = p.nfaces_along[a];
    const int fa = fid % NA, tr = fid / NA;
    int ec[3] = {0, 0, 0};
    if (DIM == 2) {
      ec[1 - a] = tr;
    } else {
      const int b0 = (a == 0) ? 1 : 0, b1 = (a == 2) ? 1 : 2;
      ec[b0] = tr % p.nel[b0];
      ec[b1] = tr / p.nel[b0];
    }
    const bool periodic = p.bc[2 * a] == 0;
    const int na = p.nel[a];
    int eL = fa - 1, eR = fa;
    if (periodic && eL < 0) eL = na - 1;
    const bool ghostL = !periodic && fa == 0;
    const bool ghostR = !periodic && fa == na;
    auto elin = [&](int ea) {
      int c[3] = {ec[0], ec[1], ec[2]};
      c[a] = ea;
      return c[0] + p.nel[0] * (c[1] + p.nel[1] * c[2]);
    };
    const size_t fsz = (size_t)(NV + NL) * P;
    const double* fsL = ghostL ? nullptr : w.face_states + ((size_t)elin(eL) * 2 * DIM + 2 * a + 1) * fsz;
    const double* fsR = ghostR ? nullptr : w.face_states + ((size_t)elin(eR) * 2 * DIM + 2 * a + 0) * fsz;
    double thL[NL], thR[NL];
    if (!ghostL) {
      for (int v = 0; v < NV; ++v) UL[v] = fsL[v * P + j];
      for (int l = 0; l < NL; ++l) thL[l] = fsL[(NV + l) * P + j];
    }
    if (!ghostR) {
      for (int v = 0; v < NV; ++v) UR[v] = fsR[v * P + j];
      for (int l = 0; l < NL; ++l) thR[l] = fsR[(NV + l) * P + j];
    }
    if (ghostL) {   // low boundary: ghost on the left built from the right state (reading R6)
      for (int v = 0; v < NV; ++v) UL[v] = UR[v];
      if (p.bc[2 * a] == 1) UL[1 + a] = -UL[1 + a];
      for (int l = 0; l < NL; ++l) thL[l] = thR[l];
    }
    if (ghostR) {
      for (int v = 0; v < NV; ++v) UR[v] = UL[v];
      if (p.bc[2 * a + 1] == 1) UR[1 + a] = -UR[1 + a];
      for (int l = 0; l < NL; ++l) thR[l] = thL[l];
    }
    for (int l = 0; l < NL; ++l) wl[l] = 0.5 * (thL[l] + thR[l]);
  } else {
    for (int v = 0; v < NV; ++v) { UL[v] = 1.0; UR[v] = 1.0; }
    for (int l = 0; l < NL; ++l) wl[l] = 0.0;
  }
  double F[NV];
  blended_flux<DIM, M>(UL, UR, wl, a, p.gamma, p.family, f, j, valid, sUL, sUR, sT, sF, sflag, F, w.counters);
  if (valid) {
    double* out = w.face_flux + ((size_t)p.face_off[a] + fid) * NV * P;
    for (int v = 0; v < NV; ++v) out[v * P + j] = F[v];
  }
}

// ---------------------------------------------------------------------------
// K3: level right-hand sides, blend and RK stage
// ---------------------------------------------------------------------------
template <int DIM, int M>
struct K3Smem {
  static constexpr int MD = Geo<DIM, M>::MD, NV = Geo<DIM, M>::NV, S = Geo<DIM, M>::S, NL = Geo<DIM, M>::NL;
  static constexpr int P = Geo<DIM, M>::P;
  static constexpr int FB = (M - 1) * NV * P;   // one face-group buffer
  static constexpr int o_su = 0;
  static constexpr int o_th = o_su + NV * MD;
  static constexpr int o_avg = o_th + NL * MD;
  static constexpr int o_alpha = o_avg + NV * S;
  static constexpr int o_beta = o_alpha + S;
  static constexpr int o_fb = o_beta + S;                 // element face fluxes [2 DIM][NV][P]
  static constexpr int o_fin = o_fb + 2 * DIM * NV * P;  // inner fluxes of one direction
  static constexpr int o_u = o_fin + FB;                  // union: face scratch (4 FB) | level scratch (3 NV MD) | reduction
  static constexpr int uni = (4 * FB > 3 * NV * MD ? 4 * FB : 3 * NV * MD);
  static constexpr int o_flag = o_u + uni;               // ints after the doubles
  static constexpr int total = o_flag + ((M - 1) * P + 1) / 2 + 1;
  static constexpr size_t bytes = sizeof(double) * total;
};

template <int DIM, int M, int N>
__device__ void level_volume(const double* su, const double* avg, const double* beta, double* ut, double* tmp,
                             double* fb, const KParams& p, int t, double* rhs) {
  constexpr int MD = ipow(M, DIM), NV = DIM + 2, S = Geo<DIM, M>::S;
  constexpr int off = s_off(M, DIM, N);
  const DevLevel& L = lev(p.family, ilog2(N));
  reconstruct<DIM, M, N>(ut, tmp, su, p.family, t);
  // beta-limited nodal values (eq. positivity-limiter-applied)
  if (t < MD) {
    const int s = sub_index<DIM, M>(t, N);
    const double b = beta[off + s];
    if (b != 1.0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) ut[v * MD + t] = (1.0 - b) * avg[v * S + off + s] + b * ut[v * MD + t];
    }
  }
  __syncthreads();
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (t < MD) {
      double q[NV], f[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) q[v] = ut[v * MD + t];
      Prim<DIM> w;
      w.load(q, p.gamma);
      flux_of<DIM>(q, w, a, f);
#pragma unroll
      for (int v = 0; v < NV; ++v) fb[v * MD + t] = f[v];
    }
    __syncthreads();
    // f x_a Dhat x_b P (x_c P), in increasing axis order after the a pass
    double* src = fb;
    double* dst = tmp;
    mode_sq<DIM, M, N, NV>(dst, src, L.Dhat, a, t);
    __syncthreads();
#pragma unroll
    for (int b = 0; b < DIM; ++b) {
      if (b == a) continue;
      double* nd = (dst == tmp) ? fb : tmp;
      mode_sq<DIM, M, N, NV>(nd, dst, L.P, b, t);
      __syncthreads();
      dst = nd;
    }
    if (t < MD) {
      const double c = ((double)M / (double)N) / p.dx[a];
#pragma unroll
      for (int v = 0; v < NV; ++v) rhs[v] += c * dst[v * MD + t];
    }
    __syncthreads();
  }
}

template <int DIM, int M>
__global__ void __launch_bounds__(Geo<DIM, M>::NT) k_update(KParams p, Work w, const double* __restrict__ us,
                                                            const double* __restrict__ u0, double* __restrict__ out,
                                                            double ark, double brk, double dt, const double* dt_dev,
                                                            int mode) {
  constexpr int MD = Geo<DIM, M>::MD, NV = Geo<DIM, M>::NV, S = Geo<DIM, M>::S, NL = Geo<DIM, M>::NL;
  constexpr int P = Geo<DIM, M>::P, NT = Geo<DIM, M>::NT;
  using L = K3Smem<DIM, M>;
  extern __shared__ double sm[];
  double* su = sm + L::o_su;
  double* th = sm + L::o_th;
  double* avg = sm + L::o_avg;
  double* alpha = sm + L::o_alpha;
  double* beta = sm + L::o_beta;
  double* fbd = sm + L::o_fb;
  double* fin = sm + L::o_fin;
  double* uni = sm + L::o_u;
  int* sflag = reinterpret_cast<int*>(sm + L::o_flag);
  const int t = threadIdx.x;
  const int e = blockIdx.x;
  const int fam = p.family;
  const double g = p.gamma;
  const double* ue = us + (size_t)e * NV * MD;
  for (int i = t; i < NV * MD; i += NT) su[i] = ue[i];
  const double* ce = w.coeffs + (size_t)e * 2 * S;
  for (int i = t; i < S; i += NT) { alpha[i] = ce[i]; beta[i] = ce[S + i]; }
  const int dec = w.decision[e];
  const int lmin = dec & 15, lmax = dec >> 4;
  // element coordinates
  int ec[3];
  ec[0] = e % p.nel[0];
  ec[1] = (e / p.nel[0]) % p.nel[1];
  ec[2] = (DIM == 3) ? e / (p.nel[0] * p.nel[1]) : 0;
  // element face fluxes
  for (int i = t; i < 2 * DIM * NV * P; i += NT) {
    const int face = i / (NV * P), r = i % (NV * P);
    const int a = face / 2, side = face % 2;
    const int NA = p.nfaces_along[a];
    int fa = ec[a] + side;
    if (p.bc[2 * a] == 0 && fa == p.nel[a]) fa = 0;
    int tr;
    if (DIM == 2) tr = ec[1 - a];
    else {
      const int b0 = (a == 0) ? 1 : 0, b1 = (a == 2) ? 1 : 2;
      tr = ec[b0] + p.nel[b0] * ec[b1];
    }
    const size_t fid = (size_t)p.face_off[a] + fa + (size_t)NA * tr;
    fbd[i] = w.face_flux[fid * NV * P + r];
  }
  __syncthreads();
  // blending weights
  if (t < MD) {
    double rest = 1.0;
#pragma unroll
    for (int l = NL - 1; l >= 1; --l) {
      const int n = 1 << l;
      const double A = alpha[s_off(M, DIM, n) + sub_index<DIM, M>(t, n)];
      th[l * MD + t] = A * rest;
      rest = rest * (1.0 - A);
    }
    th[t] = rest;
  }
  // averages of the active levels whose squeezing is active
  {
    double* red = uni;
    for (int l = (lmin > 1 ? lmin : 1); l <= lmax; ++l) {
      const int n = 1 << l;
      const int NS = ipow(M / n, DIM);
      const int off = s_off(M, DIM, n);
      const bool need = __syncthreads_or(t < NS && beta[off + t] != 1.0);
      if (!need) continue;
      if (n == 2) sub_averages<DIM, M, 2>(su, red, avg, t);
      else if (n == 4) sub_averages<DIM, M, 4>(su, red, avg, t);
      else sub_averages<DIM, M, (M >= 8 ? 8 : 4)>(su, red, avg, t);
    }
  }
  __syncthreads();
  double rhs[NL][NV];
#pragma unroll
  for (int l = 0; l < NL; ++l)
#pragma unroll
    for (int v = 0; v < NV; ++v) rhs[l][v] = 0.0;
  // levels carrying weight in this element, and the inner interfaces (1..M-1 along
  // each direction) they use: all of them for the FV level, the sub-element
  // boundaries for a DG level below M
  int used = 0;
#pragma unroll
  for (int l = 0; l < NL; ++l) used |= __syncthreads_or(t < MD && th[l * MD + t] != 0.0) ? (1 << l) : 0;
  int kmask = (used & 1) ? ((1 << M) - 2) : 0;
#pragma unroll
  for (int l = 1; l < NL - 1; ++l)
    if (used & (1 << l))
      for (int k = 1 << l; k < M; k += 1 << l) kmask |= 1 << k;
  const int nk = __popc(kmask);
  const bool need_inner = nk > 0;
  (void)lmin;
  double thv[NL];
#pragma unroll
  for (int l = 0; l < NL; ++l) thv[l] = (t < MD) ? th[l * MD + t] : 0.0;
  // surface terms and the FV level, direction by direction
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    if (need_inner) {
      constexpr int FB = K3Smem<DIM, M>::FB;
      double* sUL = uni;
      double* sUR = uni + FB;
      double* sT = uni + 2 * FB;
      double* sF = uni + 3 * FB;
      const bool valid = t < nk * P;
      const int f = valid ? t / P : 0, j = valid ? t % P : 0;
      // the f-th interface of the mask
      int k = 0;
      for (int cnt = -1; cnt < f && k < M - 1;) {
        ++k;
        if (kmask & (1 << k)) ++cnt;
      }
      double UL[NV], UR[NV], wl[NL];
      if (valid) {   // interface k lies between subcells k-1 and k along a
        int coords[3];
        coords[a] = k - 1;
        if (DIM == 2) {
          coords[1 - a] = j;
        } else {
          const int b0 = (a == 0) ? 1 : 0, b1 = (a == 2) ? 1 : 2;
          coords[b0] = j % M;
          coords[b1] = j / M;
        }
        int tL = coords[0] + M * coords[1];
        if (DIM == 3) tL += M * M * coords[2];
        const int tR = tL + stride_of<M>(a);
        blended_face_state<DIM, M>(su, th, beta, avg, tL, a, 1, fam, UL);
        blended_face_state<DIM, M>(su, th, beta, avg, tR, a, 0, fam, UR);
#pragma unroll
        for (int l = 0; l < NL; ++l) wl[l] = 0.5 * (th[l * MD + tL] + th[l * MD + tR]);
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) { UL[v] = 1.0; UR[v] = 1.0; }
#pragma unroll
        for (int l = 0; l < NL; ++l) wl[l] = 0.0;
      }
      double F[NV];
      blended_flux<DIM, M>(UL, UR, wl, a, g, fam, f, j, valid, sUL, sUR, sT, sF, sflag, F, w.counters);
      if (valid) {
#pragma unroll
        for (int v = 0; v < NV; ++v) fin[((k - 1) * NV + v) * P + j] = F[v];
      }
      __syncthreads();
    }
    if (t < MD) {
      const int c = (a == 0) ? (t % M) : (a == 1 ? (t / M) % M : t / (M * M));
      int j;
      if (DIM == 2) j = (a == 0) ? (t / M) : (t % M);
      else {
        const int cx = t % M, cy = (t / M) % M, cz = t / (M * M);
        j = (a == 0) ? (cy + M * cz) : (a == 1 ? (cx + M * cz) : (cx + M * cy));
      }
      // flux at interface k (0..M) of this subcell row
      auto flux_at = [&](int k, int v) -> double {
        if (k == 0) return fbd[((2 * a + 0) * NV + v) * P + j];
        if (k == M) return fbd[((2 * a + 1) * NV + v) * P + j];
        return fin[((k - 1) * NV + v) * P + j];
      };
      if (thv[0] != 0.0) {
        const double cfv = -((double)M / p.dx[a]);
#pragma unroll
        for (int v = 0; v < NV; ++v) rhs[0][v] += cfv * (flux_at(c + 1, v) - flux_at(c, v));
      }
#pragma unroll
      for (int l = 1; l < NL; ++l) {
        if (thv[l] == 0.0) continue;
        const int n = 1 << l;
        const int lo = (c / n) * n, i = c - lo;
        const DevLevel& Lv = lev(fam, l);
        const double cl = ((double)M / (double)n) / p.dx[a];
#pragma unroll
        for (int v = 0; v < NV; ++v)
          rhs[l][v] -= cl * (Lv.Bh0[i] * flux_at(lo, v) + Lv.Bhn[i] * flux_at(lo + n, v));
      }
    }
    __syncthreads();
  }
  // volume terms of the active DG levels
  {
    double* ut = uni;
    double* tmp = uni + NV * MD;
    double* fb = uni + 2 * NV * MD;
#pragma unroll
    for (int l = 1; l < NL; ++l) {
      if (l < lmin || l > lmax) continue;
      if (!__syncthreads_or(t < MD && thv[l] != 0.0)) continue;
      if (l == 1) level_volume<DIM, M, 2>(su, avg, beta, ut, tmp, fb, p, t, rhs[1]);
      else if (l == 2) level_volume<DIM, M, 4>(su, avg, beta, ut, tmp, fb, p, t, rhs[2]);
      else level_volume<DIM, M, (M >= 8 ? 8 : 4)>(su, avg, beta, ut, tmp, fb, p, t, rhs[NL - 1]);
    }
  }
  if (t < MD) {
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = (thv[0] != 0.0) ? thv[0] * rhs[0][v] : 0.0;
#pragma unroll
    for (int l = 1; l < NL; ++l) {
      if (thv[l] == 0.0) continue;
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += thv[l] * rhs[l][v];
    }
    double* oe = out + (size_t)e * NV * MD;
    if (mode == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) oe[v * MD + t] = acc[v];
    } else {
      const double dtv = dt_dev ? *dt_dev : dt;
      const double* u0e = u0 + (size_t)e * NV * MD;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const double us_v = su[v * MD + t];
        const double r = us_v + dtv * acc[v];
        oe[v * MD + t] = (ark != 0.0 ? ark * u0e[v * MD + t] : 0.0) + brk * r;
      }
    }
  }
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
  double rest = 1.0;
  for (int l = NL - 1; l >= 1; --l) {
    const int n = 1 << l;
    const double A = ce[s_off(M, DIM, n) + sub_index<DIM, M>(t, n)];
    thl[l] = A * rest;
    rest = rest * (1.0 - A);
  }
  thl[0] = rest;
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
// time step: max wave speed over all means (eq. euler-max-eigenvalue)
// ---------------------------------------------------------------------------
template <int DIM, int M>
__global__ void k_lambda(KParams p, Work w, const double* __restrict__ u) {
  constexpr int MD = Geo<DIM, M>::MD, NV = Geo<DIM, M>::NV;
  const size_t n = (size_t)p.E * MD;
  double lmax = 0.0;
  bool bad = false;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t e = i / MD, t = i % MD;
    const double* q0 = u + e * NV * MD + t;
    double q[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) q[v] = q0[v * MD];
    const double r = q[0];
    const double c = sqrt(p.gamma * pressure<DIM>(q, p.gamma) / r);
    double lam = fabs(q[1] / r) + c;
#pragma unroll
    for (int k = 1; k < DIM; ++k) lam = fmax(lam, fabs(q[1 + k] / r) + c);
    if (!isfinite(lam)) bad = true;
    else lmax = fmax(lmax, lam);
  }
  for (int o = 16; o > 0; o /= 2) lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  __shared__ double sw[32];
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  if (lane == 0) sw[wid] = lmax;
  if (bad) atomicOr((unsigned long long*)&w.counters[0], 2ull);
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < (int)(blockDim.x / 32); ++i) m = fmax(m, sw[i]);
    atomicMax(w.lmax, (unsigned long long)__double_as_longlong(m));
  }
}

__global__ void k_dt(KParams p, Work w, double* dt_out) {
  const double lam = __longlong_as_double((long long)*w.lmax);
  const double denom = (double)(1 << (p.dim - 1)) * (2.0 * p.M - 1.0);
  const double dt = p.cfl * p.dxmin / (denom * lam);
  *w.dt = dt;
  if (dt_out) *dt_out = dt;
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
int upload_ops(int family, int M) {
  (void)M;   // the tables of levels 2, 4, 8 do not depend on M
  DevOps ops;
  memset(&ops, 0, sizeof(ops));
  for (int l = 1; l <= 3; ++l) {
    LevelOps h;
    if (!make_level_ops(1 << l, family, &h)) return 1;
    DevLevel& d = ops.lv[l];
    memcpy(d.R, h.R, sizeof(d.R));
    memcpy(d.P, h.P, sizeof(d.P));
    memcpy(d.Dn, h.Dn, sizeof(d.Dn));
    memcpy(d.Dhat, h.Dhat, sizeof(d.Dhat));
    memcpy(d.IRf, h.IRf, sizeof(d.IRf));
    memcpy(d.Bh0, h.Bh0, sizeof(d.Bh0));
    memcpy(d.Bhn, h.Bhn, sizeof(d.Bhn));
    memcpy(d.w, h.w, sizeof(d.w));
  }
  cudaError_t err = cudaMemcpyToSymbol(c_ops, &ops, sizeof(DevOps), sizeof(DevOps) * family);
  return err == cudaSuccess ? 0 : 2;
}

namespace {

template <int DIM, int M>
int ind_impl(const KParams& p, const Work& w, const double* u, const double* frozen, cudaStream_t s) {
  constexpr size_t smem = K1Smem<DIM, M>::bytes;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_indicator<DIM, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
    attr = true;
  }
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
             double dt, const double* dt_dev, int mode, cudaStream_t s) {
  constexpr size_t smem = K3Smem<DIM, M>::bytes;
  static bool attr = false;
  if (!attr) {
    if (cudaFuncSetAttribute(k_update<DIM, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 1;
    attr = true;
  }
  k_update<DIM, M><<<p.E, Geo<DIM, M>::NT, smem, s>>>(p, w, us, u0, out, a, b, dt, dt_dev, mode);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <int DIM, int M>
int theta_impl(const KParams& p, const Work& w, double* theta, double* abar, cudaStream_t s) {
  k_theta<DIM, M><<<p.E, Geo<DIM, M>::NT, 0, s>>>(p, w, theta, abar);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

template <int DIM, int M>
int dt_impl(const KParams& p, const Work& w, const double* u, double* dt_out, cudaStream_t s) {
  if (cudaMemsetAsync(w.lmax, 0, sizeof(unsigned long long), s) != cudaSuccess) return 1;
  const size_t n = (size_t)p.E * Geo<DIM, M>::MD;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  k_lambda<DIM, M><<<blocks, 256, 0, s>>>(p, w, u);
  k_dt<<<1, 1, 0, s>>>(p, w, dt_out);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace

#define SESC_DISPATCH(FN, ...)                                           \
  do {                                                                   \
    if (p.dim == 2 && p.M == 4) return FN<2, 4>(__VA_ARGS__);            \
    if (p.dim == 2 && p.M == 8) return FN<2, 8>(__VA_ARGS__);            \
    if (p.dim == 3 && p.M == 4) return FN<3, 4>(__VA_ARGS__);            \
    if (p.dim == 3 && p.M == 8) return FN<3, 8>(__VA_ARGS__);            \
    return 1;                                                            \
  } while (0)

int launch_indicator(const KParams& p, const Work& w, const double* u, const double* frozen, void* stream) {
  SESC_DISPATCH(ind_impl, p, w, u, frozen, (cudaStream_t)stream);
}
int launch_face_flux(const KParams& p, const Work& w, void* stream) {
  SESC_DISPATCH(face_impl, p, w, (cudaStream_t)stream);
}
int launch_update(const KParams& p, const Work& w, const double* us, const double* u0, double* out, double a,
                  double b, double dt, const double* dt_dev, int mode, void* stream) {
  SESC_DISPATCH(upd_impl, p, w, us, u0, out, a, b, dt, dt_dev, mode, (cudaStream_t)stream);
}
int launch_theta(const KParams& p, const Work& w, double* theta, double* abar, void* stream) {
  SESC_DISPATCH(theta_impl, p, w, theta, abar, (cudaStream_t)stream);
}
int launch_dt(const KParams& p, const Work& w, const double* u, double* dt_out, void* stream) {
  SESC_DISPATCH(dt_impl, p, w, u, dt_out, (cudaStream_t)stream);
}

}  // namespace sesc
