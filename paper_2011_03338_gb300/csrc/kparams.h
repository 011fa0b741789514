// Parameters shared by the host launch code and the kernels (internal header).
#pragma once
#include <stdint.h>

namespace sesc {

struct KParams {
  int dim, M, E, S;
  int nel[3];
  int bc[6];
  int nfaces_along[3];   // faces along direction a per transverse element row
  int face_off[3];       // offset of direction a in the interface-flux array (in faces)
  double dx[3];
  double mdx[3];         // -M / dx[a], the flux-difference factor of the subcell scale
  double dxmin;
  double gamma, tauA, tauS, alphaH, alphaL, betaL, cfl;
  int family;
};

// Workspace pointers of a handle (device memory).
struct Work {
  double* face_states;      // [E][2*dim][nv + L][P] in the compute type (double or float)
  double* face_flux;        // [faces][nv][P] in the compute type
  double* coeffs;           // [E][2][S]
  uint8_t* decision;        // [E]
  unsigned long long* lmax; // max wave speed bits
  double* dt;               // one double
  long long* counters;      // [16]
};

// Launchers of one precision (namespaces fp64 and split, kernels in blend_kernels.cuh).
#define SESC_DECLARE_LAUNCHERS(NS)                                                                          \
  namespace NS {                                                                                            \
  int upload_ops(int family);                                                                               \
  int launch_indicator(const KParams& p, const Work& w, const double* u, const double* frozen, void* stream); \
  int launch_face_flux(const KParams& p, const Work& w, void* stream);                                      \
  int launch_update(const KParams& p, const Work& w, const double* us, const double* u0, double* out,        \
                    double a, double b, double dt, const double* dt_dev, int mode, void* stream);            \
  int launch_theta(const KParams& p, const Work& w, double* theta, double* abar, void* stream);              \
  int launch_dt(const KParams& p, const Work& w, const double* u, double* dt_out, void* stream);              \
  }
SESC_DECLARE_LAUNCHERS(fp64)
SESC_DECLARE_LAUNCHERS(split)
#undef SESC_DECLARE_LAUNCHERS

namespace fp64 {
// adjoint of uout = a u0 + b (us + dt R(us)) with the workspace's coefficients:
// us_bar = bscale * uout_bar + rscale * (dR/dus)^T uout_bar (us_bar is overwritten),
// u0_bar += ascale * uout_bar (if not null); fbe, fsb: scratch of E*2d*nv*P doubles each
int launch_stage_vjp(const KParams& p, const Work& w, const double* us, const double* uout_bar, double ascale,
                     double bscale, double rscale, double* us_bar, double* u0_bar, double* fbe, double* fsb,
                     void* stream);
}

}  // namespace sesc
