// Batched ensembles: many independent problems of uneven mesh sizes advanced
// together. Problems with the same (dim, M, precision) form a group; every group
// runs each phase of a stage (indicator + face states, interface fluxes, update)
// as one persistent grid-stride launch over the concatenated elements of all its
// problems, with each problem's own parameters, workspace and time step. Groups
// run on separate stream branches so a small group fills SMs a large one leaves
// idle. A whole SSP-RK3 step can be captured once into a CUDA graph and replayed.
// The grid size of every batched kernel (so the number of elements each CTA
// walks) is chosen by a timing autotuner over multiples of the SM count.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "../../include/sesc.h"
#include "kparams.h"

using sesc::BatchView;
using sesc::FaceTask;
using sesc::KParams;
using sesc::Work;

namespace {

struct BatchLaunchers {
  int (*upload_ops)(int);
  int (*fused)(const BatchView&, int, int, const double*, const double*, double*, double, double, int, int, unsigned*,
               long long, void*);
  int (*fused_nf)(int, int);
  int (*indicator)(const BatchView&, int, int, const double*, int, void*);
  int (*face_flux)(const BatchView&, int, int, int, void*);
  int (*update)(const BatchView&, int, int, const double*, const double*, double*, double, double, int, int, void*);
  int (*dt)(const BatchView&, int, int, const double*, int, void*);
  int (*max_blocks)(int, int, int);
};

const BatchLaunchers kBatchFP64 = {sesc::fp64::upload_ops,          sesc::fp64::launch_batch_stage_fused,
                                   sesc::fp64::fused_faces_per_task, sesc::fp64::launch_batch_indicator,
                                   sesc::fp64::launch_batch_face_flux, sesc::fp64::launch_batch_update,
                                   sesc::fp64::launch_batch_dt,     sesc::fp64::batch_max_blocks};
const BatchLaunchers kBatchSplit = {sesc::split::upload_ops,          sesc::split::launch_batch_stage_fused,
                                    sesc::split::fused_faces_per_task, sesc::split::launch_batch_indicator,
                                    sesc::split::launch_batch_face_flux, sesc::split::launch_batch_update,
                                    sesc::split::launch_batch_dt,     sesc::split::batch_max_blocks};

constexpr int kKinds = SESC_BATCH_NUM_KERNEL_KINDS;
// polls of a grid-barrier wait in the fused stage kernel before it gives up (128 ns
// apart: about 2 s), unless set with sesc_batch_set_barrier_cap
constexpr long long kBarrierCap = 1LL << 24;

int ipow_b(int b, int e) {
  int r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Group {
  int dim, M, prec;
  const BatchLaunchers* L;
  std::vector<int> probs;   // problem indices, in batch order
  int Etot, ntasks, ltiles;
  BatchView view;           // device tables
  int items[kKinds];        // work items per kernel kind
  int maxgrid[kKinds];      // all CTAs resident
  int grid[kKinds];
  bool fused;               // stages as one persistent launch (k_stage_fused)
  int fused_grid;           // its grid: all CTAs resident
  unsigned* bar;            // its grid-barrier words (2)
  cudaStream_t side;        // branch stream (groups after the first)
  cudaEvent_t fork, join;
};

}  // namespace

struct sesc_batch {
  int device;
  int nprob;
  int sms;
  std::vector<sesc_config> cfg;
  std::vector<KParams> kp;
  std::vector<Work> w;
  std::vector<long long> off;   // state offsets in doubles, nprob + 1
  std::vector<Group> groups;
  void* arena;                  // workspace and tables, one allocation
  double* stage[2];
  unsigned long long* lmax;     // [nprob][2]
  double* dt;                   // [nprob]
  long long* counters;          // [nprob][kCounters]
  long long barrier_cap;        // polls before a grid-barrier wait of the fused kernel gives up
  // captured SSP-RK3 steps, one per (u, uout, dt_dev); a time loop that swaps
  // two state buffers uses two
  struct Captured {
    const double* u;
    double* uout;
    double* dt;
    cudaGraphExec_t exec;
  };
  static constexpr int kMaxGraphs = 4;
  bool use_graph;
  cudaStream_t cap;
  std::vector<Captured> graphs;
};

namespace {

void drop_graph(sesc_batch* b) {
  for (auto& g : b->graphs) cudaGraphExecDestroy(g.exec);
  b->graphs.clear();
}

void release(sesc_batch* b) {
  drop_graph(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (Group& g : b->groups) {
    if (g.side) cudaStreamDestroy(g.side);
    if (g.fork) cudaEventDestroy(g.fork);
    if (g.join) cudaEventDestroy(g.join);
  }
  cudaFree(b->arena);
  cudaFree(b->stage[0]);
  cudaFree(b->stage[1]);
}

// the phases of one stage for one group on stream s
int group_stage(sesc_batch* b, Group& g, const double* us, const double* u0, double* out, double a, double bb,
                int mode, cudaStream_t s) {
  if (g.fused)
    return g.L->fused(g.view, g.dim, g.M, us, u0, out, a, bb, mode, g.fused_grid, g.bar, b->barrier_cap, s)
               ? SESC_ECUDA
               : SESC_OK;
  if (g.L->indicator(g.view, g.dim, g.M, us, g.grid[SESC_BATCH_KERNEL_INDICATOR], s)) return SESC_ECUDA;
  if (g.L->face_flux(g.view, g.dim, g.M, g.grid[SESC_BATCH_KERNEL_FACE_FLUX], s)) return SESC_ECUDA;
  if (g.L->update(g.view, g.dim, g.M, us, u0, out, a, bb, mode, g.grid[SESC_BATCH_KERNEL_UPDATE], s))
    return SESC_ECUDA;
  (void)b;
  return SESC_OK;
}

int group_step(sesc_batch* b, Group& g, const double* u, double* uout, cudaStream_t s) {
  if (g.L->dt(g.view, g.dim, g.M, u, g.grid[SESC_BATCH_KERNEL_DT], s)) return SESC_ECUDA;
  int rc = group_stage(b, g, u, u, b->stage[0], 0.0, 1.0, 1, s);
  if (rc == SESC_OK) rc = group_stage(b, g, b->stage[0], u, b->stage[1], 0.75, 0.25, 1, s);
  if (rc == SESC_OK) rc = group_stage(b, g, b->stage[1], u, uout, 1.0 / 3.0, 2.0 / 3.0, 1, s);
  return rc;
}

// fork the group branches off stream s, run fn(group, stream) on each, join back
template <class Fn>
int for_groups(sesc_batch* b, cudaStream_t s, Fn fn) {
  const int ng = (int)b->groups.size();
  for (int i = 1; i < ng; ++i) {
    Group& g = b->groups[i];
    if (cudaEventRecord(g.fork, s) != cudaSuccess) return SESC_ECUDA;
    if (cudaStreamWaitEvent(g.side, g.fork, 0) != cudaSuccess) return SESC_ECUDA;
  }
  int rc = SESC_OK;
  for (int i = 0; i < ng; ++i) {
    Group& g = b->groups[i];
    const int r = fn(g, i == 0 ? s : g.side);
    if (r != SESC_OK && rc == SESC_OK) rc = r;
  }
  for (int i = 1; i < ng; ++i) {
    Group& g = b->groups[i];
    if (cudaEventRecord(g.join, g.side) != cudaSuccess) return SESC_ECUDA;
    if (cudaStreamWaitEvent(s, g.join, 0) != cudaSuccess) return SESC_ECUDA;
  }
  return rc;
}

int enqueue_step(sesc_batch* b, const double* u, double* uout, double* dt_dev, cudaStream_t s) {
  if (cudaMemsetAsync(b->lmax, 0, 2 * sizeof(unsigned long long) * b->nprob, s) != cudaSuccess) return SESC_ECUDA;
  int rc = for_groups(b, s, [&](Group& g, cudaStream_t gs) { return group_step(b, g, u, uout, gs); });
  if (rc != SESC_OK) return rc;
  if (dt_dev && cudaMemcpyAsync(dt_dev, b->dt, sizeof(double) * b->nprob, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return SESC_ECUDA;
  return SESC_OK;
}

// capture one step on the internal stream; returns the executable graph or null
cudaGraphExec_t capture_step(sesc_batch* b, const double* u, double* uout, double* dt_dev, int* rc_out) {
  *rc_out = SESC_ECUDA;
  if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return nullptr;
  const int rc = enqueue_step(b, u, uout, dt_dev, b->cap);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
  if (rc != SESC_OK || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    *rc_out = rc != SESC_OK ? rc : SESC_ECUDA;
    return nullptr;
  }
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  *rc_out = SESC_OK;
  return exec;
}

}  // namespace

extern "C" {

int sesc_batch_create(const sesc_config* cfgs, int nproblems, sesc_batch** out) {
  if (!out) return SESC_EINVAL;
  *out = nullptr;
  if (!cfgs || nproblems < 1) return SESC_EINVAL;
  for (int k = 0; k < nproblems; ++k) {
    const int rc = sesc::validate_config(&cfgs[k]);
    if (rc != SESC_OK) return rc;
    for (int i = 0; i < 2 * cfgs[k].dim; ++i)
      if (cfgs[k].bc[i] == SESC_BC_HALO) return SESC_EINVAL;   // batch problems are whole meshes
  }
  sesc_batch* b = new (std::nothrow) sesc_batch();
  if (!b) return SESC_ENOMEM;
  b->nprob = nproblems;
  b->barrier_cap = kBarrierCap;
  b->cfg.assign(cfgs, cfgs + nproblems);
  if (cudaGetDevice(&b->device) != cudaSuccess) { delete b; return SESC_ECUDA; }
  if (cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
    delete b;
    return SESC_ECUDA;
  }
  b->kp.resize(nproblems);
  b->w.resize(nproblems);
  b->off.assign(nproblems + 1, 0);
  std::vector<long long> nfaces(nproblems);
  for (int k = 0; k < nproblems; ++k) {
    sesc::make_params(&cfgs[k], &b->kp[k], &nfaces[k]);
    const KParams& p = b->kp[k];
    b->off[k + 1] = b->off[k] + (long long)p.E * (p.dim + 2) * ipow_b(p.M, p.dim);
  }
  if (b->off[nproblems] > (1LL << 40)) { delete b; return SESC_EINVAL; }
  // groups by (dim, M, precision), in order of first appearance
  for (int k = 0; k < nproblems; ++k) {
    const KParams& p = b->kp[k];
    const int prec = cfgs[k].precision;
    Group* gp = nullptr;
    for (Group& g : b->groups)
      if (g.dim == p.dim && g.M == p.M && g.prec == prec) gp = &g;
    if (!gp) {
      b->groups.push_back(Group());
      gp = &b->groups.back();
      gp->dim = p.dim;
      gp->M = p.M;
      gp->prec = prec;
      gp->L = (prec == SESC_FP32_SPLIT) ? &kBatchSplit : &kBatchFP64;
    }
    gp->probs.push_back(k);
  }
  // sizes of the workspace (per problem) and of the tables (per group)
  size_t bytes = 0;
  std::vector<size_t> ws_off(nproblems);
  for (int k = 0; k < nproblems; ++k) {
    const KParams& p = b->kp[k];
    const int d = p.dim, nv = d + 2, P = ipow_b(p.M, d - 1);
    int nl = 1;
    for (int n = p.M; n >= 2; n /= 2) ++nl;
    ws_off[k] = bytes;
    bytes += align256(sizeof(double) * (size_t)p.E * 2 * d * (nv + nl) * P);
    bytes += align256(sizeof(double) * (size_t)nfaces[k] * nv * P);
    bytes += align256(sizeof(double) * (size_t)p.E * 2 * p.S);
    bytes += align256((size_t)p.E);
  }
  const size_t lmax_off = bytes;
  bytes += align256(2 * sizeof(unsigned long long) * nproblems);
  const size_t dt_off = bytes;
  bytes += align256(sizeof(double) * nproblems);
  const size_t ct_off = bytes;
  bytes += align256(sizeof(long long) * sesc::kCounters * nproblems);
  // host copies of the group tables
  struct HostTables {
    std::vector<KParams> P;
    std::vector<Work> W;
    std::vector<int> gstart, lstart;
    std::vector<long long> uoff;
    std::vector<FaceTask> tasks, tasks_f;
    size_t oP, oW, og, ol, ou, ot, of, ob;
  };
  std::vector<HostTables> ht(b->groups.size());
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    Group& g = b->groups[gi];
    HostTables& t = ht[gi];
    const int P = ipow_b(g.M, g.dim - 1);
    int NF = 128 / P;
    const int NFf = g.L->fused_nf(g.dim, g.M);
    t.gstart.push_back(0);
    t.lstart.push_back(0);
    for (size_t j = 0; j < g.probs.size(); ++j) {
      const int k = g.probs[j];
      const KParams& p = b->kp[k];
      t.gstart.push_back(t.gstart.back() + p.E);
      const long long nmeans = (long long)p.E * ipow_b(p.M, p.dim);
      t.lstart.push_back(t.lstart.back() + (int)((nmeans + sesc::kLambdaTile - 1) / sesc::kLambdaTile));
      t.uoff.push_back(b->off[k]);
      for (int a = 0; a < p.dim; ++a) {
        long long nf = p.nfaces_along[a];
        for (int c = 0; c < p.dim; ++c)
          if (c != a) nf *= p.nel[c];
        for (long long f = 0; f < nf; f += NF) t.tasks.push_back(FaceTask{(int)j, a, (int)f, (int)nf});
        for (long long f = 0; f < nf; f += NFf) t.tasks_f.push_back(FaceTask{(int)j, a, (int)f, (int)nf});
      }
    }
    g.Etot = t.gstart.back();
    g.ltiles = t.lstart.back();
    g.ntasks = (int)t.tasks.size();
    t.oP = bytes;
    bytes += align256(sizeof(KParams) * g.probs.size());
    t.oW = bytes;
    bytes += align256(sizeof(Work) * g.probs.size());
    t.og = bytes;
    bytes += align256(sizeof(int) * t.gstart.size());
    t.ol = bytes;
    bytes += align256(sizeof(int) * t.lstart.size());
    t.ou = bytes;
    bytes += align256(sizeof(long long) * t.uoff.size());
    t.ot = bytes;
    bytes += align256(sizeof(FaceTask) * t.tasks.size());
    t.of = bytes;
    bytes += align256(sizeof(FaceTask) * t.tasks_f.size());
    t.ob = bytes;
    bytes += 256;   // the fused kernel's grid-barrier words
  }
  bool ok = cudaMalloc(&b->arena, bytes) == cudaSuccess;
  ok = ok && cudaMalloc(&b->stage[0], sizeof(double) * (size_t)b->off[nproblems]) == cudaSuccess;
  ok = ok && cudaMalloc(&b->stage[1], sizeof(double) * (size_t)b->off[nproblems]) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    release(b);
    delete b;
    return SESC_ENOMEM;
  }
  unsigned char* base = static_cast<unsigned char*>(b->arena);
  b->lmax = reinterpret_cast<unsigned long long*>(base + lmax_off);
  b->dt = reinterpret_cast<double*>(base + dt_off);
  b->counters = reinterpret_cast<long long*>(base + ct_off);
  for (int k = 0; k < nproblems; ++k) {
    const KParams& p = b->kp[k];
    const int d = p.dim, nv = d + 2, P = ipow_b(p.M, d - 1);
    int nl = 1;
    for (int n = p.M; n >= 2; n /= 2) ++nl;
    unsigned char* q = base + ws_off[k];
    Work& w = b->w[k];
    w.face_states = reinterpret_cast<double*>(q);
    q += align256(sizeof(double) * (size_t)p.E * 2 * d * (nv + nl) * P);
    w.face_flux = reinterpret_cast<double*>(q);
    q += align256(sizeof(double) * (size_t)nfaces[k] * nv * P);
    w.coeffs = reinterpret_cast<double*>(q);
    q += align256(sizeof(double) * (size_t)p.E * 2 * p.S);
    w.decision = q;
    w.lmax = b->lmax + 2 * k;
    w.dt = b->dt + k;
    w.counters = b->counters + sesc::kCounters * k;
  }
  int rc = SESC_OK;
  bool uploaded[2][2] = {{false, false}, {false, false}};
  for (size_t gi = 0; gi < b->groups.size() && rc == SESC_OK; ++gi) {
    Group& g = b->groups[gi];
    HostTables& t = ht[gi];
    for (int k : g.probs) {
      t.P.push_back(b->kp[k]);
      t.W.push_back(b->w[k]);
      const int fam = b->kp[k].family;
      if (!uploaded[g.prec][fam]) {
        if (g.L->upload_ops(fam) != 0) rc = SESC_ECUDA;
        uploaded[g.prec][fam] = true;
      }
    }
    BatchView& v = g.view;
    v.P = reinterpret_cast<const KParams*>(base + t.oP);
    v.W = reinterpret_cast<const Work*>(base + t.oW);
    v.gstart = reinterpret_cast<const int*>(base + t.og);
    v.lstart = reinterpret_cast<const int*>(base + t.ol);
    v.uoff = reinterpret_cast<const long long*>(base + t.ou);
    v.ftasks = reinterpret_cast<const FaceTask*>(base + t.ot);
    v.ftasks_f = reinterpret_cast<const FaceTask*>(base + t.of);
    v.ntasks_f = (int)t.tasks_f.size();
    g.bar = reinterpret_cast<unsigned*>(base + t.ob);
    v.nprob = (int)g.probs.size();
    v.Etot = g.Etot;
    v.ntasks = g.ntasks;
    v.ltiles = g.ltiles;
    ok = cudaMemcpy(base + t.oP, t.P.data(), sizeof(KParams) * t.P.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(base + t.oW, t.W.data(), sizeof(Work) * t.W.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(base + t.og, t.gstart.data(), sizeof(int) * t.gstart.size(), cudaMemcpyHostToDevice) ==
                   cudaSuccess;
    ok = ok && cudaMemcpy(base + t.ol, t.lstart.data(), sizeof(int) * t.lstart.size(), cudaMemcpyHostToDevice) ==
                   cudaSuccess;
    ok = ok && cudaMemcpy(base + t.ou, t.uoff.data(), sizeof(long long) * t.uoff.size(), cudaMemcpyHostToDevice) ==
                   cudaSuccess;
    ok = ok && cudaMemcpy(base + t.ot, t.tasks.data(), sizeof(FaceTask) * t.tasks.size(),
                          cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(base + t.of, t.tasks_f.data(), sizeof(FaceTask) * t.tasks_f.size(),
                          cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) rc = SESC_ECUDA;
    g.items[SESC_BATCH_KERNEL_INDICATOR] = g.Etot;
    g.items[SESC_BATCH_KERNEL_FACE_FLUX] = g.ntasks;
    g.items[SESC_BATCH_KERNEL_UPDATE] = g.Etot;
    g.items[SESC_BATCH_KERNEL_DT] = g.ltiles;
    for (int kind = 0; kind < kKinds && rc == SESC_OK; ++kind) {
      const int per_sm = g.L->max_blocks(g.dim, g.M, kind);
      if (per_sm < 1) { rc = SESC_ECUDA; break; }
      g.maxgrid[kind] = per_sm * b->sms;
      g.grid[kind] = std::max(1, std::min(g.maxgrid[kind], g.items[kind]));
    }
    if (rc == SESC_OK) {
      // the fused stage kernel: all CTAs resident (a cooperative launch needs them so)
      const int per_sm = g.L->max_blocks(g.dim, g.M, 4);
      if (per_sm < 1) rc = SESC_ECUDA;
      g.fused_grid = per_sm * b->sms;
      g.fused = true;
    }
    if (rc == SESC_OK && gi > 0) {
      if (cudaStreamCreateWithFlags(&g.side, cudaStreamNonBlocking) != cudaSuccess) rc = SESC_ECUDA;
      if (cudaEventCreateWithFlags(&g.fork, cudaEventDisableTiming) != cudaSuccess) rc = SESC_ECUDA;
      if (cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming) != cudaSuccess) rc = SESC_ECUDA;
    }
  }
  if (rc == SESC_OK && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) rc = SESC_ECUDA;
  if (rc == SESC_OK && cudaMemset(b->counters, 0, sizeof(long long) * sesc::kCounters * nproblems) != cudaSuccess) rc = SESC_ECUDA;
  if (rc == SESC_OK && cudaDeviceSynchronize() != cudaSuccess) rc = SESC_ECUDA;
  if (rc != SESC_OK) {
    cudaGetLastError();
    release(b);
    delete b;
    return rc;
  }
  *out = b;
  return SESC_OK;
}

void sesc_batch_destroy(sesc_batch* b) {
  if (!b) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  release(b);
  cudaSetDevice(prev);
  delete b;
}

int sesc_batch_offsets(const sesc_batch* b, int64_t* offsets) {
  if (!b || !offsets) return SESC_EINVAL;
  for (int k = 0; k <= b->nprob; ++k) offsets[k] = (int64_t)b->off[k];
  return SESC_OK;
}

int sesc_batch_num_groups(const sesc_batch* b) { return b ? (int)b->groups.size() : -1; }

int sesc_batch_group_of(const sesc_batch* b, int k) {
  if (!b || k < 0 || k >= b->nprob) return -1;
  for (size_t gi = 0; gi < b->groups.size(); ++gi)
    for (int j : b->groups[gi].probs)
      if (j == k) return (int)gi;
  return -1;
}

int sesc_batch_rhs(sesc_batch* b, const double* u, double* dudt, void* stream) {
  if (!b || !u || !dudt || u == dudt) return SESC_EINVAL;
  return for_groups(b, (cudaStream_t)stream, [&](Group& g, cudaStream_t gs) {
    return group_stage(b, g, u, nullptr, dudt, 0.0, 1.0, 0, gs);
  });
}

int sesc_batch_dt(sesc_batch* b, const double* u, double* dt_dev, void* stream) {
  if (!b || !u) return SESC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(b->lmax, 0, 2 * sizeof(unsigned long long) * b->nprob, s) != cudaSuccess) return SESC_ECUDA;
  int rc = for_groups(b, s, [&](Group& g, cudaStream_t gs) {
    return g.L->dt(g.view, g.dim, g.M, u, g.grid[SESC_BATCH_KERNEL_DT], gs) ? SESC_ECUDA : SESC_OK;
  });
  if (rc != SESC_OK) return rc;
  if (dt_dev && cudaMemcpyAsync(dt_dev, b->dt, sizeof(double) * b->nprob, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return SESC_ECUDA;
  return SESC_OK;
}

int sesc_batch_rk3_step(sesc_batch* b, const double* u, double* uout, double* dt_dev, void* stream) {
  if (!b || !u || !uout || u == uout) return SESC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (!b->use_graph) return enqueue_step(b, u, uout, dt_dev, s);
  cudaGraphExec_t exec = nullptr;
  for (auto& g : b->graphs)
    if (g.u == u && g.uout == uout && g.dt == dt_dev) exec = g.exec;
  if (!exec) {
    int rc = SESC_OK;
    exec = capture_step(b, u, uout, dt_dev, &rc);
    if (!exec) return rc;
    if ((int)b->graphs.size() == sesc_batch::kMaxGraphs) {
      cudaGraphExecDestroy(b->graphs.front().exec);
      b->graphs.erase(b->graphs.begin());
    }
    b->graphs.push_back(sesc_batch::Captured{u, uout, dt_dev, exec});
  }
  return cudaGraphLaunch(exec, s) == cudaSuccess ? SESC_OK : SESC_ECUDA;
}

int sesc_batch_use_graph(sesc_batch* b, int enable) {
  if (!b) return SESC_EINVAL;
  b->use_graph = enable != 0;
  if (!b->use_graph) drop_graph(b);
  return SESC_OK;
}

int sesc_batch_grids(const sesc_batch* b, int32_t* grids) {
  if (!b || !grids) return SESC_EINVAL;
  for (size_t gi = 0; gi < b->groups.size(); ++gi)
    for (int kind = 0; kind < kKinds; ++kind) grids[gi * kKinds + kind] = b->groups[gi].grid[kind];
  return SESC_OK;
}

int sesc_batch_set_grids(sesc_batch* b, const int32_t* grids) {
  if (!b || !grids) return SESC_EINVAL;
  for (size_t gi = 0; gi < b->groups.size(); ++gi)
    for (int kind = 0; kind < kKinds; ++kind)
      if (grids[gi * kKinds + kind] < 1) return SESC_EINVAL;
  for (size_t gi = 0; gi < b->groups.size(); ++gi)
    for (int kind = 0; kind < kKinds; ++kind) b->groups[gi].grid[kind] = grids[gi * kKinds + kind];
  drop_graph(b);
  return SESC_OK;
}

int sesc_batch_autotune(sesc_batch* b, const double* u, int reps, void* stream) {
  if (!b || !u || reps < 1) return SESC_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  drop_graph(b);
  // one eager stage so face states, fluxes and time steps exist for every kernel
  int rc = sesc_batch_dt(b, u, nullptr, stream);
  if (rc == SESC_OK)
    rc = for_groups(b, s, [&](Group& g, cudaStream_t gs) {
      return group_stage(b, g, u, u, b->stage[0], 0.0, 1.0, 1, gs);
    });
  if (rc != SESC_OK) return rc;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return SESC_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return SESC_ECUDA;
  }
  for (Group& g : b->groups) {
    for (int kind = 0; kind < kKinds && rc == SESC_OK; ++kind) {
      // candidates: multiples of the SM count up to all CTAs resident, and one CTA per item
      std::vector<int> cand;
      for (int m = 1; m <= 64; m *= 2) {
        const int gsz = b->sms * m;
        if (gsz > g.maxgrid[kind] || gsz > g.items[kind]) break;
        cand.push_back(gsz);
      }
      cand.push_back(std::min(g.maxgrid[kind], g.items[kind]));
      cand.push_back(g.items[kind]);
      std::sort(cand.begin(), cand.end());
      cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
      float best = 1e30f;
      int best_grid = g.grid[kind];
      for (int gsz : cand) {
        auto launch = [&]() -> int {
          switch (kind) {
            case SESC_BATCH_KERNEL_INDICATOR: return g.L->indicator(g.view, g.dim, g.M, u, gsz, s);
            case SESC_BATCH_KERNEL_FACE_FLUX: return g.L->face_flux(g.view, g.dim, g.M, gsz, s);
            case SESC_BATCH_KERNEL_UPDATE:
              return g.L->update(g.view, g.dim, g.M, u, u, b->stage[0], 0.0, 1.0, 1, gsz, s);
            default: return g.L->dt(g.view, g.dim, g.M, u, gsz, s);
          }
        };
        if (launch()) { rc = SESC_ECUDA; break; }
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps; ++r)
          if (launch()) { rc = SESC_ECUDA; break; }
        cudaEventRecord(e1, s);
        if (rc != SESC_OK || cudaEventSynchronize(e1) != cudaSuccess) { rc = SESC_ECUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
          best = ms;
          best_grid = gsz;
        }
      }
      g.grid[kind] = best_grid;
    }
    // one stage as one persistent launch at 1, 2, 4 ... x SMs up to all CTAs resident,
    // against the three separate launches at their tuned grids; keep the fastest
    if (rc == SESC_OK) {
      std::vector<int> cand;
      for (int m = 1; m <= 64 && b->sms * m <= g.fused_grid; m *= 2) cand.push_back(b->sms * m);
      cand.push_back(g.fused_grid);
      std::sort(cand.begin(), cand.end());
      cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
      const int maxgrid = g.fused_grid;
      float best = 1e30f;
      int best_grid = 0;   // 0: separate launches
      for (int gsz = -1; gsz < (int)cand.size() && rc == SESC_OK; ++gsz) {
        g.fused = gsz >= 0;
        if (g.fused) g.fused_grid = cand[gsz];
        auto launch = [&]() { return group_stage(b, g, u, u, b->stage[0], 0.0, 1.0, 1, s); };
        if (launch() != SESC_OK) { rc = SESC_ECUDA; break; }
        cudaEventRecord(e0, s);
        for (int r = 0; r < reps; ++r)
          if (launch() != SESC_OK) { rc = SESC_ECUDA; break; }
        cudaEventRecord(e1, s);
        if (rc != SESC_OK || cudaEventSynchronize(e1) != cudaSuccess) { rc = SESC_ECUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
          best = ms;
          best_grid = g.fused ? g.fused_grid : 0;
        }
      }
      g.fused = best_grid > 0;
      g.fused_grid = best_grid > 0 ? best_grid : maxgrid;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != SESC_OK) return rc;
  // the repeated launches counted every non-permissible event several times
  return cudaMemsetAsync(b->counters, 0, sizeof(long long) * sesc::kCounters * b->nprob, s) == cudaSuccess &&
                 cudaStreamSynchronize(s) == cudaSuccess
             ? SESC_OK
             : SESC_ECUDA;
}

int sesc_batch_fused(const sesc_batch* b, int32_t* fused_grid) {
  if (!b || !fused_grid) return SESC_EINVAL;
  for (size_t gi = 0; gi < b->groups.size(); ++gi)
    fused_grid[gi] = b->groups[gi].fused ? b->groups[gi].fused_grid : 0;
  return SESC_OK;
}

int sesc_batch_set_fused(sesc_batch* b, const int32_t* fused_grid) {
  if (!b || !fused_grid) return SESC_EINVAL;
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    const Group& g = b->groups[gi];
    const int most = g.L->max_blocks(g.dim, g.M, 4) * b->sms;
    if (fused_grid[gi] < 0 || fused_grid[gi] > most) return SESC_EINVAL;
  }
  for (size_t gi = 0; gi < b->groups.size(); ++gi) {
    Group& g = b->groups[gi];
    g.fused = fused_grid[gi] > 0;
    if (g.fused) g.fused_grid = fused_grid[gi];
  }
  drop_graph(b);
  return SESC_OK;
}

int sesc_batch_set_barrier_cap(sesc_batch* b, int64_t polls) {
  if (!b || polls < 0) return SESC_EINVAL;
  b->barrier_cap = (long long)polls;
  drop_graph(b);
  return SESC_OK;
}

int sesc_batch_status(sesc_batch* b, int64_t* counters) {
  if (!b) return SESC_EINVAL;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  std::vector<long long> c((size_t)sesc::kCounters * b->nprob);
  cudaError_t e1 = cudaDeviceSynchronize();
  cudaError_t e2 = cudaMemcpy(c.data(), b->counters, sizeof(long long) * c.size(), cudaMemcpyDeviceToHost);
  cudaSetDevice(prev);
  if (e1 != cudaSuccess || e2 != cudaSuccess) return SESC_ECUDA;
  if (counters)
    for (int k = 0; k < b->nprob; ++k)
      for (int i = 0; i < 16; ++i) counters[16 * k + i] = (int64_t)c[(size_t)sesc::kCounters * k + i];
  long long flags = 0;
  for (int k = 0; k < b->nprob; ++k) flags |= c[(size_t)sesc::kCounters * k];
  if (flags & 8) return SESC_EBOUNDS;
  if (flags & 4) return SESC_ETIMEOUT;
  if (flags & 1) return SESC_ENONPERMISSIBLE;
  if (flags & 2) return SESC_ENONFINITE;
  return SESC_OK;
}

int sesc_batch_reset_status(sesc_batch* b, void* stream) {
  if (!b) return SESC_EINVAL;
  return cudaMemsetAsync(b->counters, 0, sizeof(long long) * sesc::kCounters * b->nprob, (cudaStream_t)stream) == cudaSuccess
             ? SESC_OK
             : SESC_ECUDA;
}

}  // extern "C"
