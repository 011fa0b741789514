// Adjoint (vector-Jacobian product) of the right-hand side and of one RK stage with
// frozen blending coefficients, written once for the compute type `real` (included
// after blend_kernels.cuh by kernels_fp64.cu and by kernels_split.cu; it uses that
// file's tables, helpers and the forward indicator kernel).
//
// With alpha, beta (and so theta) frozen, R(u) is a composition of linear maps
// (reconstruction, squeezing with fixed beta, interface interpolation, operator
// passes, the theta blend) and pointwise nonlinear maps (the Euler flux at the
// nodes, the HLL flux at interface points). The reverse pass applies the
// transposed linear maps in reverse order and the transposed Jacobians of the
// pointwise maps: the Euler flux's in reverse mode written out, the HLL flux's from
// forward-mode dual numbers through the same templated physics as the forward
// kernels (branches of HLL, min / max of the Einfeldt speeds and the
// permissibility fallback follow the forward state).
//
// Every adjoint value is formed by gathering: each output (a flux adjoint at an
// interface, the adjoint of a mean) is summed by one thread in a fixed order from
// the values that feed it, so the result is the same bit for bit from run to run
// (no floating-point atomics). With real = float the transposed flux differences
// and their theta weights (the forward's FP64 islands) and the stage combination
// are formed in FP64; the rest in FP32.
//
// kernels (one stage): Kt3 k_update_vjp (element): level and FV flux differences,
// volume operators, limited reconstruction, inner interfaces -> u_bar (part) and
// the adjoints of the element-face fluxes; Kt2 k_face_flux_vjp (face): candidate
// and HLL reverse -> adjoints of the element-face states; Kt1 k_face_state_vjp
// (element): reverse of the blended element-face states -> u_bar (rest) and the
// stage combination.

namespace sesc {
namespace SESC_NS {

// ---------------------------------------------------------------------------
// dual numbers (value, derivative) for pointwise Jacobians; their arithmetic is
// found by argument-dependent lookup from the templated physics
// ---------------------------------------------------------------------------
namespace ad {
template <typename T>
struct Dual {
  T v, d;
  __device__ __forceinline__ Dual() : v(0), d(0) {}
  __device__ __forceinline__ Dual(T x) : v(x), d(0) {}
  __device__ __forceinline__ Dual(T x, T y) : v(x), d(y) {}
};
template <typename T>
__device__ __forceinline__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return Dual<T>(a.v + b.v, a.d + b.d); }
template <typename T>
__device__ __forceinline__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return Dual<T>(a.v - b.v, a.d - b.d); }
template <typename T>
__device__ __forceinline__ Dual<T> operator*(Dual<T> a, Dual<T> b) { return Dual<T>(a.v * b.v, a.d * b.v + a.v * b.d); }
template <typename T>
__device__ __forceinline__ Dual<T> operator/(Dual<T> a, Dual<T> b) {
  const T q = a.v / b.v;
  return Dual<T>(q, (a.d - q * b.d) / b.v);
}
template <typename T>
__device__ __forceinline__ Dual<T> operator-(Dual<T> a) { return Dual<T>(-a.v, -a.d); }
template <typename T>
__device__ __forceinline__ bool operator>=(Dual<T> a, Dual<T> b) { return a.v >= b.v; }
template <typename T>
__device__ __forceinline__ bool operator<=(Dual<T> a, Dual<T> b) { return a.v <= b.v; }
template <typename T>
__device__ __forceinline__ Dual<T> fma(Dual<T> a, Dual<T> b, Dual<T> c) { return a * b + c; }
template <typename T>
__device__ __forceinline__ Dual<T> sqrt(Dual<T> a) {
  const T s = ::sqrt(a.v);
  return Dual<T>(s, s > T(0) ? a.d / (T(2) * s) : T(0));
}
template <typename T>
__device__ __forceinline__ Dual<T> fmax(Dual<T> a, Dual<T> b) { return a.v >= b.v ? a : b; }
template <typename T>
__device__ __forceinline__ Dual<T> fmin(Dual<T> a, Dual<T> b) { return a.v <= b.v ? a : b; }
}  // namespace ad
typedef ad::Dual<real> Dual;

// Reverse mode of the Euler flux (flux_of_t), written out with v = m / rho and
// p = (g - 1)(E - m.v / 2): one evaluation of the primitives, then their adjoints.

// qbar += J(q)^T over the primitives: the adjoints vb of v, pb of p and invb of
// 1/rho (w: the primitives of q)
template <int DIM>
__device__ __forceinline__ void prim_vjp(const real* q, const PrimT<real, DIM>& w, real g, const real* vb, real pb,
                                         real invb, real* qbar) {
  constexpr int NV = DIM + 2;
  const real gm1 = g - real(1);
  qbar[NV - 1] += gm1 * pb;
  const real kinb = real(-0.5) * gm1 * pb;   // kin = m.v
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const real vbk = vb[k] + kinb * q[1 + k];
    qbar[1 + k] += kinb * w.v[k] + vbk * w.inv;
    invb += vbk * q[1 + k];
  }
  qbar[0] -= invb * w.inv * w.inv;
}

// qbar += sum_a J_a(q)^T fbar_a over the directions a (Euler flux)
template <int DIM>
__device__ void flux_vjp(const real* q, const real (*fbar)[DIM + 2], real g, real* qbar) {
  constexpr int NV = DIM + 2;
  PrimT<real, DIM> w;
  w.load(q, g);
  real vb[DIM], pb = 0;
#pragma unroll
  for (int k = 0; k < DIM; ++k) vb[k] = 0;
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    const real* fb = fbar[a];
    real vab = fb[NV - 1] * (q[NV - 1] + w.p);
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      vab = fma(fb[1 + k], q[1 + k], vab);
      qbar[1 + k] += fb[1 + k] * w.v[a];
    }
    vb[a] += vab;
    pb += fb[1 + a] + fb[NV - 1] * w.v[a];
    qbar[1 + a] += fb[0];
    qbar[NV - 1] += fb[NV - 1] * w.v[a];
  }
  prim_vjp<DIM>(q, w, g, vb, pb, real(0), qbar);
}

// (uLbar, uRbar) += J_HLL(uL, uR)^T Fbar
template <int DIM>
__device__ void hll_vjp(const real* uL, const real* uR, int a, real g, const real* Fbar, real* uLbar, real* uRbar) {
  constexpr int NV = DIM + 2;
#pragma unroll 1
  for (int k = 0; k < 2 * NV; ++k) {
    Dual dL[NV], dR[NV], F[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      dL[v] = Dual(uL[v], k == v ? real(1) : real(0));
      dR[v] = Dual(uR[v], k == NV + v ? real(1) : real(0));
    }
    hll_t<Dual, DIM>(dL, dR, a, Dual(g), F);
    real s = 0;
#pragma unroll
    for (int v = 0; v < NV; ++v) s = fma(Fbar[v], F[v].d, s);
    if (k < NV) uLbar[k] += s;
    else uRbar[k - NV] += s;
  }
}

// transposed blockwise n-mode product along axis a: out[v][t] = sum_j A[j][i] in[v][t + (j - i) stride]
template <int DIM, int M, int N, int NVV>
__device__ __forceinline__ void mode_sq_t(real* out, const real* in, const real* A, int a, int t) {
  constexpr int MD = ipow(M, DIM);
  if (t >= MD) return;
  const int st = stride_of<M>(a);
  const int i = coord_of<M>(t, a) % N;
  const int base = t - i * st;
#pragma unroll
  for (int v = 0; v < NVV; ++v) {
    real s = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) s = fma(A[j * N + i], in[v * MD + base + j * st], s);
    out[v * MD + t] = s;
  }
}

// transposed transverse operator on a group of faces (mirror of `transverse`)
template <int DIM, int M, int N>
__device__ __forceinline__ void transverse_t(const real* src, real* sT, const real* A, int f, int j, bool valid,
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
        for (int k = 0; k < N; ++k) s = fma(A[k * N + i], src[(f * NV + v) * P + base + k], s);
        out[v] = s;
      }
    }
  } else {
    // forward: along b0 (stride 1) then b1 (stride M); transposed: b1 first, then b0
    if (valid) {
      const int i1 = (j / M) % N, b1 = j - i1 * M;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        real s = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) s = fma(A[k * N + i1], src[(f * NV + v) * P + b1 + k * M], s);
        sT[(f * NV + v) * P + j] = s;
      }
    }
    __syncthreads();
    if (valid) {
      const int i0 = (j % M) % N, b0 = j - i0;
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        real s = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) s = fma(A[k * N + i0], sT[(f * NV + v) * P + b0 + k], s);
        out[v] = s;
      }
    }
    __syncthreads();
  }
}

// reverse of one level candidate of blended_flux: given the adjoint Fb of the
// blended flux at this point, accumulate into ULb / URb (and into F1b where the
// candidate fell back to the FV flux). Scratch as in blended_flux.
template <int DIM, int M, int N>
__device__ void level_candidate_vjp(real wl, const real* Fb, int a, real g, int family, int f, int j, bool valid,
                                    real* sUL, real* sUR, real* sT, real* sF, int* sflag, real* F1b, real* ULb,
                                    real* URb) {
  constexpr int NV = DIM + 2;
  constexpr int P = ipow(M, DIM - 1);
  const DevLevel& L = lev(family, ilog2(N));
  real rL[NV], rR[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) { rL[v] = real(1); rR[v] = real(1); }
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
  // adjoint of P (.) P^T: the candidate's weight times Fb, transposed P along the transverse axes
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) sF[(f * NV + v) * P + j] = (blk && wl != real(0)) ? wl * Fb[v] : real(0);
  }
  __syncthreads();
  real Hb[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) Hb[v] = real(0);
  transverse_t<DIM, M, N>(sF, sT, L.P, f, j, valid, Hb);
  real rLb[NV], rRb[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) { rLb[v] = real(0); rRb[v] = real(0); }
  if (blk) hll_vjp<DIM>(rL, rR, a, g, Hb, rLb, rRb);
  // transposed reconstruction back to the face states
  __syncthreads();
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) sF[(f * NV + v) * P + j] = rLb[v];
  }
  __syncthreads();
  real t1[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) t1[v] = real(0);
  transverse_t<DIM, M, N>(sF, sT, L.R, f, j, valid, t1);
  __syncthreads();
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      ULb[v] += t1[v];
      sF[(f * NV + v) * P + j] = rRb[v];
    }
  }
  __syncthreads();
  transverse_t<DIM, M, N>(sF, sT, L.R, f, j, valid, t1);
  if (valid) {
#pragma unroll
    for (int v = 0; v < NV; ++v) URb[v] += t1[v];
    if (!blk && wl != real(0)) {
#pragma unroll
      for (int v = 0; v < NV; ++v) F1b[v] += wl * Fb[v];
    }
  }
  __syncthreads();
}

// reverse of blended_flux: ULb, URb = adjoints of the face states for the flux adjoint
// Fb. Ends with a barrier: the scratch arrays are free for the caller afterwards.
template <int DIM, int M>
__device__ void blended_flux_vjp(const real* UL, const real* UR, const real* w, const real* Fb, int a, real g,
                                 int family, int f, int j, bool valid, real* sUL, real* sUR, real* sT, real* sF,
                                 int* sflag, real* ULb, real* URb) {
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
  real F1b[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    ULb[v] = real(0);
    URb[v] = real(0);
    F1b[v] = (valid && w[0] != real(0)) ? w[0] * Fb[v] : real(0);
  }
  __syncthreads();
#pragma unroll
  for (int l = 1; l < NL; ++l) {
    if (!__syncthreads_or(valid && w[l] != real(0))) continue;
    if (l == 1)
      level_candidate_vjp<DIM, M, 2>(w[l], Fb, a, g, family, f, j, valid, sUL, sUR, sT, sF, sflag, F1b, ULb, URb);
    else if (l == 2)
      level_candidate_vjp<DIM, M, 4>(w[l], Fb, a, g, family, f, j, valid, sUL, sUR, sT, sF, sflag, F1b, ULb, URb);
    else
      level_candidate_vjp<DIM, M, (M >= 8 ? 8 : 4)>(w[l], Fb, a, g, family, f, j, valid, sUL, sUR, sT, sF, sflag,
                                                     F1b, ULb, URb);
  }
  if (valid) {
    bool any = false;
#pragma unroll
    for (int v = 0; v < NV; ++v) any = any || F1b[v] != real(0);
    if (any) hll_vjp<DIM>(UL, UR, a, g, F1b, ULb, URb);
  }
  __syncthreads();
}

// Reverse of the blended face states (reading R1), gathered at subcell t: every face
// state along direction a that depends on t's mean lies on t's row along a inside
// t's level-n sub-element (the level-n polynomial's interface value uses the n means
// of that row) or is one of t's own two faces (the FV part theta^(1) u_t). Fs(k, side,
// v) gives the adjoint of the state at interface k (0..M) on `side` (0: the left face
// state of subcell k, 1: the right face state of subcell k - 1), zero for faces not in
// the set handled. Adds into ub[NV]; the part through the sub-element averages (beta
// < 1) of t's own face states goes to pa[l - 1][v] (summed per sub-element later).
template <int DIM, int M, class FaceAdj>
__device__ __forceinline__ void face_state_gather(const real* th, const real* beta_s, int t, int a, int family,
                                                  const FaceAdj& Fs, real* ub, real (*pa)[DIM + 2]) {
  constexpr int MD = ipow(M, DIM);
  constexpr int NV = DIM + 2;
  constexpr int NL = ilog2(M) + 1;
  const int c = coord_of<M>(t, a);
  const int st = stride_of<M>(a);
  const real th1 = th[t];
  if (th1 != real(0)) {
#pragma unroll
    for (int v = 0; v < NV; ++v) ub[v] += th1 * (Fs(c + 1, 1, v) + Fs(c, 0, v));
  }
#pragma unroll
  for (int l = 1; l < NL; ++l) {
    const int n = 1 << l;
    const int jj = c % n, lo = c - jj;
    const int s = sub_index<DIM, M>(t, n);
    const real b = beta_s[s_off(M, DIM, n) + s];
    const real* IRf = lev(family, l).IRf;
    for (int i = 0; i < n; ++i) {
      const real thi = th[l * MD + t + (i - jj) * st];
      if (thi == real(0)) continue;
      const real cf = thi * b;
      const real wr = IRf[(i + 1) * n + jj], wl = IRf[i * n + jj];
#pragma unroll
      for (int v = 0; v < NV; ++v) ub[v] += cf * (wr * Fs(lo + i + 1, 1, v) + wl * Fs(lo + i, 0, v));
    }
    const real tht = th[l * MD + t];
    if (tht != real(0) && b != real(1)) {
      const real cf = tht * (real(1) - b);
#pragma unroll
      for (int v = 0; v < NV; ++v) pa[l - 1][v] += cf * (Fs(c + 1, 1, v) + Fs(c, 0, v));
    }
  }
}

// ub[t] += the adjoints of the sub-element averages: pa holds each subcell's
// contribution to its level-n sub-element's average adjoint; summed per sub-element
// in a fixed order (sub_reduce) and spread back divided by the sub-element's size.
// bmask: levels (bit l) with a squeezed sub-element somewhere in the element (block-uniform).
template <int DIM, int M>
__device__ void average_adjoints(real (*pa)[DIM + 2], real* red, real* avs, int bmask, int t, real* ub) {
  constexpr int MD = ipow(M, DIM), NV = DIM + 2, NL = ilog2(M) + 1;
#pragma unroll
  for (int l = 1; l < NL; ++l) {
    if (!(bmask & (1 << l))) continue;
    const int n = 1 << l;
    real x[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) x[v] = (t < MD) ? pa[l - 1][v] : real(0);
    __syncthreads();
    real r;
    if (n == 2) r = sub_reduce<DIM, M, 2, NV, false>(x, red, t);
    else if (n == 4) r = sub_reduce<DIM, M, 4, NV, false>(x, red, t);
    else r = sub_reduce<DIM, M, (M >= 8 ? 8 : 4), NV, false>(x, red, t);
    const int NS = ipow(M / n, DIM);
    if (t < NS * NV) avs[t] = r;     // [v][s]
    __syncthreads();
    if (t < MD) {
      const int s = sub_index<DIM, M>(t, n);
      const real inv = real(1) / real(ipow(n, DIM));
#pragma unroll
      for (int v = 0; v < NV; ++v) ub[v] += inv * avs[v * NS + s];
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Kt3: reverse of the update kernel (mode 0, dudt = R)
// ---------------------------------------------------------------------------
template <int DIM, int M>
struct KT3Smem {
  static constexpr int MD = Geo<DIM, M>::MD, NV = Geo<DIM, M>::NV, S = Geo<DIM, M>::S, NL = Geo<DIM, M>::NL;
  static constexpr int P = Geo<DIM, M>::P;
  static constexpr int FB = (M - 1) * NV * P;
  // doubles: r = theta * (-M/dx) * Rbar of one (level, direction), the FP64 island
  static constexpr int d_rr = 0;
  static constexpr int d_total = NV * MD;
  // reals
  static constexpr int r_su = 0;
  static constexpr int r_th = r_su + NV * MD;
  static constexpr int r_avg = r_th + NL * MD;
  static constexpr int r_beta = r_avg + NV * S;
  static constexpr int r_fbe = r_beta + S;                  // adjoints of the element-face fluxes
  static constexpr int r_fbi = r_fbe + 2 * DIM * NV * P;     // adjoints of the inner fluxes, every direction
  static constexpr int r_u = r_fbi + DIM * FB;               // union: face scratch (4 FB) | level scratch (3 NV MD)
  static constexpr int uni = (4 * FB > 3 * NV * MD ? 4 * FB : 3 * NV * MD);
  static constexpr int r_total = r_u + uni;
  static constexpr int i_flag = (M - 1) * P;
  static constexpr size_t bytes = sizeof(double) * d_total + sizeof(real) * r_total + sizeof(int) * i_flag;
};

template <int DIM, int M>
__device__ __forceinline__ int transverse_index(int t, int a) {
  if (DIM == 2) return (a == 0) ? (t / M) : (t % M);
  const int cx = t % M, cy = (t / M) % M, cz = t / (M * M);
  return (a == 0) ? (cy + M * cz) : (a == 1 ? (cx + M * cz) : (cx + M * cy));
}

// flux adjoint slot of interface k (0..M) along a at transverse point j
template <int DIM, int M>
__device__ __forceinline__ real* fbar_slot(real* fbe, real* fbi_a, int a, int k, int v, int j) {
  constexpr int NV = DIM + 2;
  constexpr int P = ipow(M, DIM - 1);
  if (k == 0) return &fbe[((2 * a + 0) * NV + v) * P + j];
  if (k == M) return &fbe[((2 * a + 1) * NV + v) * P + j];
  return &fbi_a[((k - 1) * NV + v) * P + j];
}

// reverse of one DG level along a (mirror of level_fluxes). With r_c = theta_c (-M/dx)
// Rbar_c: the interior subcell fluxes G_{lo+i+1} = c0_i F_lo + cn_i F_{lo+N} - W_i / N
// get Gbar = r_{lo+i} - r_{lo+i+1}; the sub-element boundary fluxes F_lo, F_{lo+N} get
// -r_lo + sum_i c0_i Gbar_i and r_{lo+N-1} + sum_i cn_i Gbar_i. The thread of the first
// subcell of each sub-element adds both contributions of the interface on its left
// (its own sub-element's and its left neighbour's), the last subcell's thread the
// element's right face: one writer per slot.
template <int DIM, int M, int N>
__device__ void level_fluxes_vjp(real* tmp, real* fb, double* rr, real* fbe, real* fbi_a, const KParams& p, int a,
                                 int t, double thc, const double* rb, real (*fbar)[DIM + 2]) {
  constexpr int MD = ipow(M, DIM), NV = DIM + 2;
  const DevLevel& L = lev(p.family, ilog2(N));
  const bool act = t < MD;
  const int st = stride_of<M>(a);
  const int c = act ? coord_of<M>(t, a) : 0;
  const int i = c % N, lo = c - i;
  const int j = transverse_index<DIM, M>(t, a);
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) rr[v * MD + t] = thc * rb[v];
  }
  __syncthreads();
  if (act) {
    const int t0 = t - i * st;   // first subcell of this sub-element's row
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double* r = rr + v * MD;
      tmp[v * MD + t] = (i < N - 1) ? (real)(-(r[t] - r[t + st]) / (double)N) : real(0);
      if (i == 0) {
        double s = -r[t0];
        for (int q = 0; q < N - 1; ++q) s += (double)L.c0[q] * (r[t0 + q * st] - r[t0 + (q + 1) * st]);
        if (lo > 0) {
          const int tl = t0 - N * st;
          s += r[tl + (N - 1) * st];
          for (int q = 0; q < N - 1; ++q) s += (double)L.cn[q] * (r[tl + q * st] - r[tl + (q + 1) * st]);
        }
        *fbar_slot<DIM, M>(fbe, fbi_a, a, lo, v, j) += (real)s;
      }
      if (c == M - 1) {
        double s = r[t];
        for (int q = 0; q < N - 1; ++q) s += (double)L.cn[q] * (r[t0 + q * st] - r[t0 + (q + 1) * st]);
        *fbar_slot<DIM, M>(fbe, fbi_a, a, M, v, j) += (real)s;
      }
    }
  }
  __syncthreads();
  // W = f x_a C x_b P (b ascending): transposed in reverse order
  real* src = tmp;
  real* dst = fb;
#pragma unroll
  for (int b = DIM - 1; b >= 0; --b) {
    if (b == a) continue;
    mode_sq_t<DIM, M, N, NV>(dst, src, L.P, b, t);
    __syncthreads();
    real* x = src;
    src = dst;
    dst = x;
  }
  // fbar_a[j'] = sum_{k < N-1} C[k][j'] Wbar[k]
  if (act) {
    const int base = t - i * st;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      real s = 0;
#pragma unroll
      for (int k = 0; k < N - 1; ++k) s = fma(L.C[k * N + i], src[v * MD + base + k * st], s);
      fbar[a][v] = s;
    }
  }
  __syncthreads();
}

// reverse of one DG level: flux adjoints of every direction, nodal Jacobians, the
// transposed limited reconstruction into ub (and the average part into pa)
template <int DIM, int M, int N>
__device__ void level_vjp(const real* su, const real* avg, const real* beta, real* ut, real* tmp, real* fb,
                          double* rr, real* fbe, real* fbi, const KParams& p, int t, double thl, const double* rb,
                          real* ub, real* pa) {
  constexpr int MD = ipow(M, DIM), NV = DIM + 2, P = ipow(M, DIM - 1);
  constexpr int FB = (M - 1) * NV * P;
  constexpr int off = s_off(M, DIM, N);
  const DevLevel& L = lev(p.family, ilog2(N));
  limited_nodal<DIM, M, N>(su, avg, beta, ut, tmp, p, t);
  real fbar[DIM][DIM + 2];
  // keep the nodal values of this thread: the passes below reuse ut's scratch
  real q[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) q[v] = (t < MD) ? ut[v * MD + t] : real(1);
#pragma unroll
  for (int a = 0; a < DIM; ++a)
    level_fluxes_vjp<DIM, M, N>(tmp, fb, rr, fbe, fbi + a * FB, p, a, t, p.mdx[a] * thl, rb, fbar);
  real utb[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) utb[v] = real(0);
  if (t < MD && thl != 0.0) flux_vjp<DIM>(q, fbar, (real)p.gamma, utb);
  // limited values (1 - beta) <u> + beta u~: beta part through the transposed reconstruction
  const int s = (t < MD) ? sub_index<DIM, M>(t, N) : 0;
  const real b = (t < MD) ? beta[off + s] : real(1);
  if (t < MD) {
#pragma unroll
    for (int v = 0; v < NV; ++v) ut[v * MD + t] = b * utb[v];
  }
  __syncthreads();
  // u~ = u x_0 R x_1 R (x_2 R): transposed passes in reverse order
  real* src = ut;
  real* dst = tmp;
#pragma unroll
  for (int a = DIM - 1; a >= 0; --a) {
    mode_sq_t<DIM, M, N, NV>(dst, src, L.R, a, t);
    __syncthreads();
    real* x = src;
    src = dst;
    dst = x;
  }
  if (t < MD) {
#pragma unroll
    for (int v = 0; v < NV; ++v) ub[v] += src[v * MD + t];
    if (b != real(1)) {
#pragma unroll
      for (int v = 0; v < NV; ++v) pa[v] += (real(1) - b) * utb[v];
    }
  }
  __syncthreads();
}

// face adjoints of the inner interfaces of one direction pass, stored per face slot
// (popcount of the interface mask below k) in sUL (side 1) and sUR (side 0)
template <int DIM, int M>
struct InnerFaces {
  const real* sL;
  const real* sR;
  int kmask, j;
  __device__ __forceinline__ real operator()(int k, int side, int v) const {
    constexpr int NV = DIM + 2, P = ipow(M, DIM - 1);
    if (k <= 0 || k >= M || !((kmask >> k) & 1)) return real(0);
    const int f = __popc(kmask & ((1 << k) - 1));
    return (side ? sL : sR)[(f * NV + v) * P + j];
  }
};

template <int DIM, int M>
__global__ void __launch_bounds__(Geo<DIM, M>::NT) k_update_vjp(KParams p, Work w, const double* __restrict__ us,
                                                                const double* __restrict__ rbar, double rscale,
                                                                double* __restrict__ ubar_out, real* fbe_out) {
  constexpr int MD = Geo<DIM, M>::MD, NV = Geo<DIM, M>::NV, S = Geo<DIM, M>::S, NL = Geo<DIM, M>::NL;
  constexpr int P = Geo<DIM, M>::P, NT = Geo<DIM, M>::NT;
  constexpr int FB = KT3Smem<DIM, M>::FB;
  using L = KT3Smem<DIM, M>;
  extern __shared__ double sm[];
  double* rr = sm + L::d_rr;
  real* rs = reinterpret_cast<real*>(sm + L::d_total);
  real* su = rs + L::r_su;
  real* th = rs + L::r_th;
  real* avg = rs + L::r_avg;
  real* beta = rs + L::r_beta;
  real* fbe = rs + L::r_fbe;
  real* fbi = rs + L::r_fbi;
  real* uni = rs + L::r_u;
  int* sflag = reinterpret_cast<int*>(rs + L::r_total);
  const int t = threadIdx.x;
  const int e = blockIdx.x;
  const int fam = p.family;
  const real g = (real)p.gamma;
  const double* ue = us + (size_t)e * NV * MD;
  for (int i = t; i < NV * MD; i += NT) su[i] = (real)ue[i];
  const double* ce = w.coeffs + (size_t)e * 2 * S;
  for (int i = t; i < S; i += NT) beta[i] = (real)ce[S + i];
  for (int i = t; i < 2 * DIM * NV * P; i += NT) fbe[i] = real(0);
  for (int i = t; i < DIM * FB; i += NT) fbi[i] = real(0);
  // blending weights: FP64 per thread for the flux-difference factors (as the forward
  // update kernel), and in the compute type for face states and level tests
  double thv[NL];
  if (t < MD) {
    weights_of<DIM, M>(ce, t, thv);
    real rest = 1;
#pragma unroll
    for (int l = NL - 1; l >= 1; --l) {
      const int n = 1 << l;
      const real A = (real)ce[s_off(M, DIM, n) + sub_index<DIM, M>(t, n)];
      th[l * MD + t] = A * rest;
      rest = rest * (real(1) - A);
    }
    th[t] = rest;
  } else {
#pragma unroll
    for (int l = 0; l < NL; ++l) thv[l] = 0.0;
  }
  __syncthreads();
  int used = 0;
#pragma unroll
  for (int l = 0; l < NL; ++l) used |= __syncthreads_or(t < MD && th[l * MD + t] != real(0)) ? (1 << l) : 0;
  int kmask = (used & 1) ? ((1 << M) - 2) : 0;
#pragma unroll
  for (int l = 1; l < NL - 1; ++l)
    if (used & (1 << l))
      for (int k = 1 << l; k < M; k += 1 << l) kmask |= 1 << k;
  const int nk = __popc(kmask);
  int bmask = 0;   // used levels with a squeezed sub-element
#pragma unroll
  for (int l = 1; l < NL; ++l) {
    if (!(used & (1 << l))) continue;
    const int n = 1 << l;
    const int NS = ipow(M / n, DIM);
    const int off = s_off(M, DIM, n);
    if (!__syncthreads_or(t < NS && beta[off + t] != real(1))) continue;
    bmask |= 1 << l;
    if (n == 2) sub_averages<DIM, M, 2>(su, uni, avg, t);
    else if (n == 4) sub_averages<DIM, M, 4>(su, uni, avg, t);
    else sub_averages<DIM, M, (M >= 8 ? 8 : 4)>(su, uni, avg, t);
  }
  __syncthreads();
  double rb[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) rb[v] = (t < MD) ? rscale * rbar[(size_t)e * NV * MD + v * MD + t] : 0.0;
  real ub[NV];
  real pa[NL - 1][NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    ub[v] = real(0);
#pragma unroll
    for (int l = 0; l < NL - 1; ++l) pa[l][v] = real(0);
  }
  // FV level: R_c += theta1_c (-M/dx) (F_{c+1} - F_c): Fbar_k += r_{k-1} - r_k
  if (used & 1) {
#pragma unroll 1
    for (int a = 0; a < DIM; ++a) {
      const bool act = t < MD;
      if (act) {
        const double r0 = p.mdx[a] * thv[0];
#pragma unroll
        for (int v = 0; v < NV; ++v) rr[v * MD + t] = r0 * rb[v];
      }
      __syncthreads();
      if (act) {
        const int c = coord_of<M>(t, a), st = stride_of<M>(a);
        const int j = transverse_index<DIM, M>(t, a);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const double* r = rr + v * MD;
          *fbar_slot<DIM, M>(fbe, fbi + a * FB, a, c, v, j) += (real)((c > 0 ? r[t - st] : 0.0) - r[t]);
          if (c == M - 1) *fbar_slot<DIM, M>(fbe, fbi + a * FB, a, M, v, j) += (real)r[t];
        }
      }
      __syncthreads();
    }
  }
  // DG levels
  {
    real* ut = uni;
    real* tmp = uni + NV * MD;
    real* fb = uni + 2 * NV * MD;
#pragma unroll
    for (int l = 1; l < NL; ++l) {
      if (!(used & (1 << l))) continue;
      if (l == 1) level_vjp<DIM, M, 2>(su, avg, beta, ut, tmp, fb, rr, fbe, fbi, p, t, thv[1], rb, ub, pa[0]);
      else if (l == 2) level_vjp<DIM, M, 4>(su, avg, beta, ut, tmp, fb, rr, fbe, fbi, p, t, thv[2], rb, ub, pa[1]);
      else
        level_vjp<DIM, M, (M >= 8 ? 8 : 4)>(su, avg, beta, ut, tmp, fb, rr, fbe, fbi, p, t, thv[NL - 1], rb, ub,
                                            pa[NL - 2]);
    }
  }
  __syncthreads();
  // inner interfaces, one direction per pass: reverse of the blended flux, then of the
  // blended face states (gathered per subcell)
#pragma unroll 1
  for (int a = 0; a < DIM; ++a) {
    if (nk == 0) break;
    real* sUL = uni;
    real* sUR = uni + FB;
    real* sT = uni + 2 * FB;
    real* sF = uni + 3 * FB;
    const bool valid = t < nk * P;
    const int f = valid ? t / P : 0, j = valid ? t % P : 0;
    int k = 0;
    for (int cnt = -1; cnt < f && k < M - 1;) {
      ++k;
      if (kmask & (1 << k)) ++cnt;
    }
    real UL[NV], UR[NV], wl[NL], Fb[NV];
    if (valid) {
      const int tL = subcell_of<DIM, M>(a, k - 1, j);
      const int tR = tL + stride_of<M>(a);
      blended_face_state<DIM, M>(su, th, beta, avg, tL, a, 1, fam, UL);
      blended_face_state<DIM, M>(su, th, beta, avg, tR, a, 0, fam, UR);
#pragma unroll
      for (int l = 0; l < NL; ++l) wl[l] = real(0.5) * (th[l * MD + tL] + th[l * MD + tR]);
#pragma unroll
      for (int v = 0; v < NV; ++v) Fb[v] = fbi[a * FB + ((k - 1) * NV + v) * P + j];
    } else {
#pragma unroll
      for (int v = 0; v < NV; ++v) { UL[v] = real(1); UR[v] = real(1); Fb[v] = real(0); }
#pragma unroll
      for (int l = 0; l < NL; ++l) wl[l] = real(0);
    }
    real ULb[NV], URb[NV];
    blended_flux_vjp<DIM, M>(UL, UR, wl, Fb, a, g, fam, f, j, valid, sUL, sUR, sT, sF, sflag, ULb, URb);
    if (valid) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        sUL[(f * NV + v) * P + j] = ULb[v];
        sUR[(f * NV + v) * P + j] = URb[v];
      }
    }
    __syncthreads();
    if (t < MD) {
      const InnerFaces<DIM, M> Fs{sUL, sUR, kmask, transverse_index<DIM, M>(t, a)};
      face_state_gather<DIM, M>(th, beta, t, a, fam, Fs, ub, pa);
    }
    __syncthreads();
  }
  average_adjoints<DIM, M>(pa, uni, uni + NV * MD, bmask, t, ub);
  if (t < MD) {
    double* uo = ubar_out + (size_t)e * NV * MD;
#pragma unroll
    for (int v = 0; v < NV; ++v) uo[v * MD + t] = (double)ub[v];
  }
  real* fo = fbe_out + (size_t)e * 2 * DIM * NV * P;
  for (int i = t; i < 2 * DIM * NV * P; i += NT) fo[i] = fbe[i];
}

// ---------------------------------------------------------------------------
// Kt2: reverse of the interface flux at element faces
// ---------------------------------------------------------------------------
template <int DIM, int M>
__global__ void __launch_bounds__(128) k_face_flux_vjp(KParams p, Work w, int a, int nfaces, const real* fbe,
                                                      real* fsb) {
  constexpr int NV = Geo<DIM, M>::NV, NL = Geo<DIM, M>::NL, P = Geo<DIM, M>::P;
  constexpr int NF = FaceCfg<DIM, M>::NF;
  __shared__ real sUL[NF * NV * P], sUR[NF * NV * P], sT[NF * NV * P], sF[NF * NV * P];
  __shared__ int sflag[NF * P];
  const int tid = threadIdx.x;
  const int f = tid / P, j = tid % P;
  const int fid = blockIdx.x * NF + f;
  const bool valid = fid < nfaces;
  const real* fstates = reinterpret_cast<const real*>(w.face_states);
  real UL[NV], UR[NV], wl[NL], Fb[NV];
  int eL = -1, eR = -1;
  bool ghostL = false, ghostR = false;
  if (valid) {
    const int NA = p.nfaces_along[a];
    const int fa = fid % NA, tr = fid / NA;
    const bool periodic = p.bc[2 * a] == 0;
    const int na = p.nel[a];
    int xL = fa - 1, xR = fa;
    if (periodic && xL < 0) xL = na - 1;
    ghostL = !periodic && fa == 0;
    ghostR = !periodic && fa == na;
    auto elin = [&](int ea) { return (int)chk(element_of<DIM>(p, a, ea, tr), p.E, w.counters); };
    const size_t fsz = (size_t)(NV + NL) * P;
    const size_t esz = (size_t)2 * DIM * NV * P;
    real thL[NL], thR[NL];
#pragma unroll
    for (int v = 0; v < NV; ++v) Fb[v] = real(0);
    if (!ghostL) {
      eL = elin(xL);
      const real* fsL = fstates + ((size_t)eL * 2 * DIM + 2 * a + 1) * fsz;
      for (int v = 0; v < NV; ++v) UL[v] = fsL[v * P + j];
      for (int l = 0; l < NL; ++l) thL[l] = fsL[(NV + l) * P + j];
      for (int v = 0; v < NV; ++v) Fb[v] += fbe[(size_t)eL * esz + ((2 * a + 1) * NV + v) * P + j];
    }
    if (!ghostR) {
      eR = elin(xR);
      const real* fsR = fstates + ((size_t)eR * 2 * DIM + 2 * a + 0) * fsz;
      for (int v = 0; v < NV; ++v) UR[v] = fsR[v * P + j];
      for (int l = 0; l < NL; ++l) thR[l] = fsR[(NV + l) * P + j];
      for (int v = 0; v < NV; ++v) Fb[v] += fbe[(size_t)eR * esz + ((2 * a + 0) * NV + v) * P + j];
    }
    if (ghostL) {
      for (int v = 0; v < NV; ++v) UL[v] = UR[v];
      if (p.bc[2 * a] == 1)
#pragma unroll
        for (int k = 0; k < DIM; ++k)
          if (a == k) UL[1 + k] = -UL[1 + k];
      for (int l = 0; l < NL; ++l) thL[l] = thR[l];
    }
    if (ghostR) {
      for (int v = 0; v < NV; ++v) UR[v] = UL[v];
      if (p.bc[2 * a + 1] == 1)
#pragma unroll
        for (int k = 0; k < DIM; ++k)
          if (a == k) UR[1 + k] = -UR[1 + k];
      for (int l = 0; l < NL; ++l) thR[l] = thL[l];
    }
    for (int l = 0; l < NL; ++l) wl[l] = real(0.5) * (thL[l] + thR[l]);
  } else {
    for (int v = 0; v < NV; ++v) { UL[v] = real(1); UR[v] = real(1); Fb[v] = real(0); }
    for (int l = 0; l < NL; ++l) wl[l] = real(0);
  }
  real ULb[NV], URb[NV];
  blended_flux_vjp<DIM, M>(UL, UR, wl, Fb, a, (real)p.gamma, p.family, f, j, valid, sUL, sUR, sT, sF, sflag, ULb,
                           URb);
  if (valid) {
    // a ghost state is a (mirrored) copy of the interior one: fold its adjoint back
    if (ghostL) {
      if (p.bc[2 * a] == 1)
#pragma unroll
        for (int k = 0; k < DIM; ++k)
          if (a == k) ULb[1 + k] = -ULb[1 + k];
      for (int v = 0; v < NV; ++v) URb[v] += ULb[v];
    }
    if (ghostR) {
      if (p.bc[2 * a + 1] == 1)
#pragma unroll
        for (int k = 0; k < DIM; ++k)
          if (a == k) URb[1 + k] = -URb[1 + k];
      for (int v = 0; v < NV; ++v) ULb[v] += URb[v];
    }
    const size_t esz = (size_t)2 * DIM * NV * P;
    if (!ghostL) {
      for (int v = 0; v < NV; ++v) fsb[(size_t)eL * esz + ((2 * a + 1) * NV + v) * P + j] = ULb[v];
    }
    if (!ghostR) {
      for (int v = 0; v < NV; ++v) fsb[(size_t)eR * esz + ((2 * a + 0) * NV + v) * P + j] = URb[v];
    }
  }
}

// face adjoints of the two element faces along a (fsb of this element): interface 0
// (left face state of subcell 0) and interface M (right face state of subcell M - 1)
template <int DIM, int M>
struct ElementFaces {
  const real* fe;   // [2 DIM][NV][P] of this element
  int a, j;
  __device__ __forceinline__ real operator()(int k, int side, int v) const {
    constexpr int NV = DIM + 2, P = ipow(M, DIM - 1);
    if (k == 0 && side == 0) return fe[((2 * a + 0) * NV + v) * P + j];
    if (k == M && side == 1) return fe[((2 * a + 1) * NV + v) * P + j];
    return real(0);
  }
};

// ---------------------------------------------------------------------------
// Kt1: reverse of the element-face states; adds to u_bar and finishes the stage
// adjoint: us_bar = bscale * uout_bar + (u_bar of R); u0_bar += ascale * uout_bar
// ---------------------------------------------------------------------------
template <int DIM, int M>
__global__ void __launch_bounds__(Geo<DIM, M>::NT) k_face_state_vjp(KParams p, Work w, const real* fsb,
                                                                    const double* uout_bar, double ascale,
                                                                    double bscale, double* us_bar, double* u0_bar) {
  constexpr int MD = Geo<DIM, M>::MD, NV = Geo<DIM, M>::NV, S = Geo<DIM, M>::S, NL = Geo<DIM, M>::NL;
  constexpr int P = Geo<DIM, M>::P;
  __shared__ real th[NL * MD];
  __shared__ real beta[S];
  __shared__ real red[NV * MD];
  __shared__ real avs[NV * ipow(M / 2, DIM)];
  const int t = threadIdx.x;
  const int e = blockIdx.x;
  const double* ce = w.coeffs + (size_t)e * 2 * S;
  for (int i = t; i < S; i += Geo<DIM, M>::NT) beta[i] = (real)ce[S + i];
  if (t < MD) {
    real rest = 1;
#pragma unroll
    for (int l = NL - 1; l >= 1; --l) {
      const int n = 1 << l;
      const real A = (real)ce[s_off(M, DIM, n) + sub_index<DIM, M>(t, n)];
      th[l * MD + t] = A * rest;
      rest = rest * (real(1) - A);
    }
    th[t] = rest;
  }
  __syncthreads();
  int bmask = 0;
#pragma unroll
  for (int l = 1; l < NL; ++l) {
    const int n = 1 << l;
    const int NS = ipow(M / n, DIM);
    if (__syncthreads_or(t < NS && beta[s_off(M, DIM, n) + t] != real(1))) bmask |= 1 << l;
  }
  real ub[NV];
  real pa[NL - 1][NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    ub[v] = real(0);
#pragma unroll
    for (int l = 0; l < NL - 1; ++l) pa[l][v] = real(0);
  }
  const real* fe = fsb + (size_t)e * 2 * DIM * NV * P;
  if (t < MD) {
#pragma unroll 1
    for (int a = 0; a < DIM; ++a) {
      const ElementFaces<DIM, M> Fs{fe, a, transverse_index<DIM, M>(t, a)};
      face_state_gather<DIM, M>(th, beta, t, a, p.family, Fs, ub, pa);
    }
  }
  average_adjoints<DIM, M>(pa, red, avs, bmask, t, ub);
  if (t < MD) {
    const size_t o = (size_t)e * NV * MD;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const size_t i = o + v * MD + t;
      const double ob = uout_bar[i];
      us_bar[i] = fma(bscale, ob, us_bar[i] + (double)ub[v]);
      if (u0_bar) u0_bar[i] += ascale * ob;
    }
  }
}

// ---------------------------------------------------------------------------
// launcher: adjoint of one stage uout = a u0 + b (us + dt R(us)) with the
// coefficients the preceding forward indicator launch left in the workspace
// ---------------------------------------------------------------------------
namespace detail {

template <int DIM, int M>
int vjp_impl(const KParams& p, const Work& w, const double* us, const double* uout_bar, double ascale, double bscale,
             double rscale, double* us_bar, double* u0_bar, double* fbe, double* fsb, cudaStream_t s) {
  constexpr size_t smem = KT3Smem<DIM, M>::bytes;
  static std::atomic<unsigned long long> attr{0};
  if (!smem_attr_once(k_update_vjp<DIM, M>, smem, attr)) return 1;
  real* fbe_r = reinterpret_cast<real*>(fbe);
  real* fsb_r = reinterpret_cast<real*>(fsb);
  k_update_vjp<DIM, M><<<p.E, Geo<DIM, M>::NT, smem, s>>>(p, w, us, uout_bar, rscale, us_bar, fbe_r);
  if (cudaGetLastError() != cudaSuccess) return 1;
  constexpr int NF = FaceCfg<DIM, M>::NF;
  for (int a = 0; a < DIM; ++a) {
    int nf = p.nfaces_along[a];
    for (int b = 0; b < DIM; ++b)
      if (b != a) nf *= p.nel[b];
    k_face_flux_vjp<DIM, M><<<(nf + NF - 1) / NF, 128, 0, s>>>(p, w, a, nf, fbe_r, fsb_r);
    if (cudaGetLastError() != cudaSuccess) return 1;
  }
  k_face_state_vjp<DIM, M><<<p.E, Geo<DIM, M>::NT, 0, s>>>(p, w, fsb_r, uout_bar, ascale, bscale, us_bar, u0_bar);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

}  // namespace detail

int launch_stage_vjp(const KParams& p, const Work& w, const double* us, const double* uout_bar, double ascale,
                     double bscale, double rscale, double* us_bar, double* u0_bar, double* fbe, double* fsb,
                     void* stream) {
  cudaStream_t s = (cudaStream_t)stream;
  if (p.dim == 2 && p.M == 4) return detail::vjp_impl<2, 4>(p, w, us, uout_bar, ascale, bscale, rscale, us_bar, u0_bar, fbe, fsb, s);
  if (p.dim == 2 && p.M == 8) return detail::vjp_impl<2, 8>(p, w, us, uout_bar, ascale, bscale, rscale, us_bar, u0_bar, fbe, fsb, s);
  if (p.dim == 3 && p.M == 4) return detail::vjp_impl<3, 4>(p, w, us, uout_bar, ascale, bscale, rscale, us_bar, u0_bar, fbe, fsb, s);
  if (p.dim == 3 && p.M == 8) return detail::vjp_impl<3, 8>(p, w, us, uout_bar, ascale, bscale, rscale, us_bar, u0_bar, fbe, fsb, s);
  return 1;
}

}  // namespace SESC_NS
}  // namespace sesc
