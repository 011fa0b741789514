// Parameters shared by the host launch code and the kernels (internal header).
#pragma once
#include <stdint.h>

#include "../../include/sesc.h"

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
  int single_level;      // 1: single-level DG/FV scheme (levels 1 and M only)
  int fp32_filter;       // FP64 build: 1 lets the indicator decide levels by its certified FP32 pass
  long long stage_cap;   // polls of an element's staging copy before a kernel gives up
  long long nfaces;      // interface count of all directions (rows of the face-flux array)
};

// default of KParams::stage_cap; also the bound of the second wait that lets a copy
// land before a CTA that gave up moves on
constexpr long long kStageWaitCap = 1LL << 22;

// Device counters per problem: the 16 that sesc_status reports, then one count per
// level mask (bit l set: level 2^l carries weight in the element), read by
// sesc_level_counts.
constexpr int kCounters = 32;

// Workspace pointers of a handle (device memory).
struct Work {
  double* face_states;      // [E][2*dim][nv + L][P] in the compute type (double or float)
  double* face_flux;        // [faces][nv][P] in the compute type
  double* coeffs;           // [E][2][S]
  uint8_t* decision;        // [E]
  unsigned long long* lmax; // [2]: max wave speed bits (FP64), FP32 estimate bits
  double* dt;               // one double
  long long* counters;      // [kCounters]: [0, 16) as sesc_status reports them, [16 + m] elements with level mask m
  const void* halo[6];      // per side with a SESC_BC_HALO boundary: the neighbour's packed face states (compute type)
  // element order of the update kernel (nullable): K1 appends each element to the list
  // of its level mask, K3 takes its elements class by class, so that the CTAs resident
  // on an SM at a time mostly run one code path; K1 takes its elements in the order the
  // last K3 took (read from `order`, one load per CTA)
  int* class_count;         // [16], zeroed before each K1 launch
  int* class_list;          // [16][E]
  int* order;               // [E] (nullable): the element order K3 took last (a permutation); K1 follows it
};

// Extra terms of a generalised RK stage, uout = a u0 + c u2 + b (us + g dt R(us)):
// u2 (nullable) with its coefficient c, and the factor g on dt (1 for SSP-RK3).
struct StageTerm {
  const double* u2;
  double c, g;
};

// Problems of one batch group (same dimension, M and precision), device arrays:
// P, W per problem; gstart[nprob + 1] group-local element prefix; uoff[k] the
// offset (in doubles) of problem k in the concatenated state; ftasks[ntasks] face
// tasks; lstart[nprob + 1] prefix of wave-speed tiles (kLambdaTile means each).
struct FaceTask {
  int prob, dir, first, nfaces;   // faces first .. first + NF - 1 of the nfaces along dir
};
constexpr int kLambdaTile = 4096;
struct BatchView {
  const KParams* P;
  const Work* W;
  const int* gstart;
  const long long* uoff;
  const FaceTask* ftasks;
  const int* lstart;
  int nprob, Etot, ntasks, ltiles;
  const FaceTask* ftasks_f;   // face tasks of the fused stage kernel (its block's faces per task)
  int ntasks_f;
};

// host helpers of the C ABI (sesc_abi.cu)
int validate_config(const sesc_config* cfg);
void make_params(const sesc_config* cfg, KParams* out, long long* nfaces_total);

// Launchers of one precision (namespaces fp64 and split, kernels in blend_kernels.cuh).
#define SESC_DECLARE_LAUNCHERS(NS)                                                                          \
  namespace NS {                                                                                            \
  int upload_ops(int family);                                                                               \
  int launch_indicator(const KParams& p, const Work& w, const double* u, const double* frozen, void* stream); \
  int launch_face_flux(const KParams& p, const Work& w, void* stream);                                      \
  int launch_update(const KParams& p, const Work& w, const double* us, const double* u0, double* out,        \
                    double a, double b, double dt, const double* dt_dev, int mode, void* stream);            \
  int launch_theta(const KParams& p, const Work& w, double* theta, double* abar, void* stream);              \
  int launch_pack_halo(const KParams& p, const Work& w, int a, int side, void* dst, void* stream);          \
  int launch_dt(const KParams& p, const Work& w, const double* u, double* dt_out, void* stream);              \
  int launch_update_x(const KParams& p, const Work& w, const double* us, const double* u0, double* out,      \
                      double a, double b, double dt, const double* dt_dev, const StageTerm& x, void* stream); \
  int launch_batch_indicator(const BatchView& b, int dim, int M, const double* u, int grid, void* stream);    \
  int launch_batch_face_flux(const BatchView& b, int dim, int M, int grid, void* stream);                    \
  int launch_batch_update(const BatchView& b, int dim, int M, const double* us, const double* u0, double* out, \
                          double a, double bb, int mode, int grid, void* stream);                            \
  int launch_batch_dt(const BatchView& b, int dim, int M, const double* u, int grid, void* stream);          \
  int batch_max_blocks(int dim, int M, int kind);                                                            \
  int launch_batch_stage_fused(const BatchView& b, int dim, int M, const double* us, const double* u0,      \
                               double* out, double a, double bb, int mode, int grid, unsigned* bar,        \
                               long long cap, void* stream);                                              \
  int fused_faces_per_task(int dim, int M);                                                                \
  int launch_stage_vjp(const KParams& p, const Work& w, const double* us, const double* uout_bar, double ascale, \
                       double bscale, double rscale, double* us_bar, double* u0_bar, double* fbe, double* fsb,    \
                       void* stream);                                                                        \
  }
SESC_DECLARE_LAUNCHERS(fp64)
SESC_DECLARE_LAUNCHERS(split)
#undef SESC_DECLARE_LAUNCHERS

// launch_stage_vjp: adjoint of uout = a u0 + b (us + dt R(us)) with the workspace's
// coefficients: us_bar = bscale * uout_bar + rscale * (dR/dus)^T uout_bar (us_bar is
// overwritten), u0_bar += ascale * uout_bar (if not null); fbe, fsb: scratch of
// E*2d*nv*P doubles each (used in the compute type).

}  // namespace sesc
