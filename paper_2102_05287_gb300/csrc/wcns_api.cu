// Host side of the C ABI declared in include/wcns.h: handle, scratch
// buffers, time-step control and the SSPRK3 orchestration of the sweeps.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "../../include/wcns.h"
#include "wcns_internal.h"

using namespace wcns;

struct wcns_handle {
  int ndim, nf;
  int n[3];
  long long N;
  double dx[3], inv_dx[3];
  int bc[3][2];
  double dirichlet[3][2][7];
  double *dir_face[3][2];  // optional per-face Dirichlet states (device, [nf][face cells])
  EosConst eos;
  wcns_options opt;
  cudaStream_t stream;
  double *W1, *W2, *L, *Wh;  // stage states, RHS accumulator, host-API state
  // node cache of the mixed path in 2D/3D (p, 1/rho: FP64; c, certification
  // bits: 32-bit), one entry per cell, carved from one allocation
  double *node_p, *node_ir;
  float *node_c;
  unsigned int *node_ok;
  double *trace_W1, *trace_W2;  // optional copies of the stage states
  StepCtl *ctl;
  DevStats *stats;
  long long launches;
  // CUDA-graph replay of whole SSPRK3 steps on a private stream
  cudaStream_t launch_stream;  // stream the launchers use (the caller's, or cap)
  cudaStream_t cap;
  cudaEvent_t ev_in, ev_out;
  cudaGraphExec_t graph;
  double *graph_W, *graph_t1, *graph_t2;
  double graph_dt, graph_cfl;
  int use_graphs;
  // per-kernel timing
  int prof_cap, prof_n;
  long long prof_dropped;
  cudaEvent_t *prof_ev;  // 2 * prof_cap events
  int *prof_dir;
};

namespace {

// ---------------------------------------------------------------------------
// Device helpers.
// ---------------------------------------------------------------------------
// max over cells of (|u_d| + c) (Sec. 3.3) into ctl->smax[slot][d].
__global__ void reduce_wavespeed_kernel(const double *__restrict__ W, long long N, int ndim,
                                        EosConst e, StepCtl *ctl, int slot) {
  double smax[3] = {0.0, 0.0, 0.0};
  const int E = 2 + ndim, A = 3 + ndim;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (long long)gridDim.x * blockDim.x) {
    double m[3], sp[3];
    for (int j = 0; j < ndim; ++j) m[j] = W[(2 + j) * N + i];
    state_wavespeeds(W[i], W[N + i], m, W[E * N + i], W[A * N + i], ndim, e, sp);
    for (int j = 0; j < ndim; ++j) smax[j] = (sp[j] > smax[j] || sp[j] != sp[j]) ? sp[j] : smax[j];
  }
  for (int j = 0; j < ndim; ++j) {
    unsigned long long b = __double_as_longlong(smax[j]);
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, b, o);
      b = ob > b ? ob : b;
    }
    if ((threadIdx.x & 31) == 0 && b) atomicMax(&ctl->smax[slot][j], b);
  }
}

// The uniform Dirichlet ghost states of a handle, passed BY VALUE as a
// kernel argument (no device copy, no host-to-device transfer).
struct UniformBcStates {
  double w[6][7];  // conservative states, [face][field]
  int count;
};

// max(|u_d| + c) of the uniform Dirichlet states into ctl->smax[0][d]; one
// thread per state.
__global__ void bc_wavespeed_kernel(const UniformBcStates u, int ndim, EosConst e, StepCtl *ctl) {
  const int k = threadIdx.x;
  if (k >= u.count) return;
  const double *w = u.w[k];
  double sp[3];
  state_wavespeeds(w[0], w[1], w + 2, w[2 + ndim], w[3 + ndim], ndim, e, sp);
  for (int j = 0; j < ndim; ++j) {
    // as in the reduction: NaN bits order above every finite wave speed's
    const unsigned long long b = __double_as_longlong(sp[j]);
    if (b) atomicMax(&ctl->smax[0][j], b);
  }
}

__global__ void init_ctl_kernel(StepCtl *ctl, const DevStats *stats, double t, double t_end) {
  ctl->stat0[0] = stats->inadmissible;
  ctl->stat0[1] = stats->nonfinite;
  for (int k = 0; k < 4; ++k)
    for (int d = 0; d < 3; ++d) ctl->smax[k][d] = ctl->smax_bc[d];
  ctl->dt = 0.0;
  ctl->t = t;
  ctl->t_end = t_end;
  ctl->steps = 0;
  ctl->active = t < t_end ? 1 : 0;
}

// Start of a step: take max(|u_d|+c) of W^n (left in smax[3] by the previous
// step's last combine or by a reduction), choose dt (fixed, or CFL / sum_d
// tau_d, Sec. 3.3), clip to t_end, and clear the accumulators of the stages.
__global__ void step_begin_kernel(StepCtl *ctl, int ndim, double ix0, double ix1, double ix2,
                                  double dt_fixed, double cfl, int advance_time) {
  const double ix[3] = {ix0, ix1, ix2};
  double tsum = 0.0;
  for (int d = 0; d < 3; ++d) {
    ctl->smax[0][d] = ctl->smax[3][d];
    if (d < ndim) tsum += __longlong_as_double(ctl->smax[0][d]) * ix[d];
  }
  for (int k = 1; k < 4; ++k)
    for (int d = 0; d < 3; ++d) ctl->smax[k][d] = ctl->smax_bc[d];
  double dt = dt_fixed > 0.0 ? dt_fixed : cfl / tsum;
  if (!advance_time) {
    ctl->dt = dt;
    ctl->active = 1;
    return;
  }
  if (!ctl->active || !(ctl->t < ctl->t_end)) {
    ctl->active = 0;
    ctl->dt = 0.0;
    return;
  }
  if (ctl->t + dt >= ctl->t_end) {
    dt = ctl->t_end - ctl->t;
    ctl->t = ctl->t_end;
  } else {
    ctl->t = ctl->t + dt;
  }
  ctl->dt = dt;
  ctl->steps += 1;
}

// ---------------------------------------------------------------------------
// Host helpers.
// ---------------------------------------------------------------------------
int cuda_status(cudaError_t e) { return e == cudaSuccess ? WCNS_OK : WCNS_E_CUDA; }

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) return WCNS_E_CUDA; \
  } while (0)

int launch_reduce(wcns_handle *h, const double *W, int slot) {
  const int threads = 256;
  long long blocks = (h->N + threads - 1) / threads;
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  reduce_wavespeed_kernel<<<(int)blocks, threads, 0, h->launch_stream>>>(W, h->N, h->ndim, h->eos, h->ctl, slot);
  h->launches++;
  return cuda_status(cudaGetLastError());
}

int launch_init(wcns_handle *h, double t, double t_end) {
  init_ctl_kernel<<<1, 1, 0, h->launch_stream>>>(h->ctl, h->stats, t, t_end);
  h->launches++;
  return cuda_status(cudaGetLastError());
}

int launch_begin(wcns_handle *h, double dt_fixed, double cfl, int advance_time) {
  step_begin_kernel<<<1, 1, 0, h->launch_stream>>>(h->ctl, h->ndim, h->inv_dx[0], h->inv_dx[1], h->inv_dx[2],
                                            dt_fixed, cfl, advance_time);
  h->launches++;
  return cuda_status(cudaGetLastError());
}

// The k-th sweep direction of an RHS evaluation: x, y, z in FP64; in the
// mixed path the order of mixed_first_dir (z, y, x by default).
int sweep_dir(const wcns_handle *h, int k) {
  const bool rev = h->opt.precision == WCNS_MIXED && mixed_first_dir(h->ndim) != 0;
  return rev ? h->ndim - 1 - k : k;
}

SweepArgs base_args(wcns_handle *h, int d) {
  SweepArgs a;
  memset(&a, 0, sizeof(a));
  for (int k = 0; k < 3; ++k) {
    a.n[k] = h->n[k];
    a.inv_dx_all[k] = h->inv_dx[k];
  }
  a.ncell = h->N;
  a.bc_lo = h->bc[d][0];
  a.bc_hi = h->bc[d][1];
  for (int q = 0; q < 7; ++q) {
    a.dir_lo[q] = h->dirichlet[d][0][q];
    a.dir_hi[q] = h->dirichlet[d][1][q];
  }
  a.dir_face_lo = h->dir_face[d][0];
  a.dir_face_hi = h->dir_face[d][1];
  a.face_n = h->N / h->n[d];
  a.inv_dx = h->inv_dx[d];
  a.eos = h->eos;
  a.tol.eps_ar = h->opt.eps_ar;
  a.tol.eps_a = h->opt.eps_a;
  a.tol.eps_rc = h->opt.eps_rc;
  a.tol.hs_ar = h->opt.hs_ar;
  a.tol.hs_a = h->opt.hs_a;
  a.tol.hs_rc = h->opt.hs_rc;
  set_cert(a.tol);
  a.eps_is = h->opt.eps_is;
  a.eps_is32 = (float)fmax(h->opt.eps_is, 1e-30);
  a.scheme = h->opt.scheme;
  a.ctl = h->ctl;
  a.stats = h->stats;
  a.accum_scale = h->inv_dx[d];
  a.l_unit = 1.0;
  // mixed path, 2D/3D: the first sweep of an RHS fills the node cache, the
  // later ones (same stage input) read it
  if (h->node_p && h->opt.precision == WCNS_MIXED && h->ndim > 1) {
    a.node_p = h->node_p;
    a.node_ir = h->node_ir;
    a.node_c = h->node_c;
    a.node_ok = h->node_ok;
    a.node_write = d == sweep_dir(h, 0);
    a.node_read = !a.node_write;
  }
  return a;
}

int launch_sweep(wcns_handle *h, int d, const SweepArgs &a) {
  int slot = -1;
  if (h->prof_cap > 0) {
    if (h->prof_n < h->prof_cap) {
      slot = h->prof_n++;
      h->prof_dir[slot] = d;
      cudaEventRecord(h->prof_ev[2 * slot], h->stream);
    } else {
      h->prof_dropped++;
    }
  }
  cudaError_t e = h->opt.precision == WCNS_MIXED ? launch_sweep_mixed(h->ndim, d, a, h->launch_stream)
                                                 : launch_sweep_fp64(h->ndim, d, a, h->launch_stream);
  if (slot >= 0) cudaEventRecord(h->prof_ev[2 * slot + 1], h->stream);
  h->launches++;
  return cuda_status(e);
}

void profile_free(wcns_handle *h) {
  if (h->prof_ev) {
    for (int k = 0; k < 2 * h->prof_cap; ++k) cudaEventDestroy(h->prof_ev[k]);
    free(h->prof_ev);
    free(h->prof_dir);
  }
  h->prof_ev = NULL;
  h->prof_dir = NULL;
  h->prof_cap = h->prof_n = 0;
  h->prof_dropped = 0;
}

// dW/dt of W into L for every direction (stage 0 lambda).
int enqueue_rhs(wcns_handle *h, const double *W, double *L) {
  for (int k = 0; k < h->ndim; ++k) {
    const int d = sweep_dir(h, k);
    SweepArgs a = base_args(h, d);
    a.epilogue = k == 0 ? EPI_WRITE : EPI_ACCUM;
    a.stage = 0;
    a.W_in = W;
    a.L = L;
    int st = launch_sweep(h, d, a);
    if (st) return st;
  }
  return WCNS_OK;
}

// One SSPRK3 step in place on W (Shu-Osher form, Sec. 5.3):
//   W1 = W + dt L(W);  W2 = 3/4 W + 1/4 (W1 + dt L(W1));
//   W  = 1/3 W + 2/3 (W2 + dt L(W2)).
int enqueue_step(wcns_handle *h, double *W, double dt_fixed, double cfl) {
  int st = launch_begin(h, dt_fixed, cfl, 1);
  if (st) return st;
  const double ra[3] = {0.0, 0.75, 1.0 / 3.0};
  const double rb[3] = {1.0, 0.25, 2.0 / 3.0};
  for (int s = 0; s < 3; ++s) {
    const double *Win = s == 0 ? W : (s == 1 ? h->W1 : h->W2);
    double *Wout = s == 0 ? h->W1 : (s == 1 ? h->W2 : W);
    const int d0 = sweep_dir(h, 0);
    for (int k = 0; k < h->ndim; ++k) {
      const int d = sweep_dir(h, k);
      SweepArgs a = base_args(h, d);
      a.stage = s;
      a.W_in = Win;
      a.Wn = W;
      a.L = h->L;
      // mixed path: L holds the first sweep's raw flux difference plus the
      // other directions' differences scaled by dx_d0/dx_d; the combine
      // applies 1/dx_d0 (one FP64 multiply per field less in the first sweep)
      const bool raw = h->opt.precision == WCNS_MIXED && h->ndim > 1;
      if (k < h->ndim - 1) {
        a.epilogue = k == 0 ? EPI_WRITE : EPI_ACCUM;
        a.l_raw = raw && k == 0;
        if (raw && k > 0) a.accum_scale = h->inv_dx[d] / h->inv_dx[d0];
      } else {
        a.epilogue = EPI_COMBINE;
        a.read_L = h->ndim > 1;
        a.l_unit = raw ? h->inv_dx[d0] : 1.0;
        a.rk_a = ra[s];
        a.rk_b = rb[s];
        a.W_out = Wout;
      }
      st = launch_sweep(h, d, a);
      if (st) return st;
    }
    double *trace = s == 0 ? h->trace_W1 : (s == 1 ? h->trace_W2 : NULL);
    if (trace && cudaMemcpyAsync(trace, Wout, sizeof(double) * (size_t)h->nf * (size_t)h->N,
                                 cudaMemcpyDeviceToDevice, h->launch_stream) != cudaSuccess)
      return WCNS_E_CUDA;
  }
  return WCNS_OK;
}

void drop_graph(wcns_handle *h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = NULL;
  h->graph_W = NULL;
}

// Dirichlet ghost states enter the boundary midpoints' fluxes like cells, so
// their max(|u_d| + c) bounds dt too (Sec. 3.3).  They are reduced into
// slot 0 of the (reset) step control, and the result is kept as the floor
// every wave-speed slot starts from.  Uniform states travel by value in the
// kernel's arguments; per-face states are reduced from their device copies.
// Called when the boundary data change; every entry point re-initialises
// the step control afterwards.  Stream-ordered; no allocation and no host
// memory read by the device.
int update_bc_wavespeed(wcns_handle *h) {
  cudaStream_t st = h->stream;
  cudaError_t e = cudaMemsetAsync(h->ctl, 0, sizeof(StepCtl), st);
  UniformBcStates u;
  memset(&u, 0, sizeof(u));
  for (int d = 0; d < h->ndim && e == cudaSuccess; ++d) {
    for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
      if (h->bc[d][s] != WCNS_BC_DIRICHLET) continue;
      const double *src = h->dir_face[d][s];
      if (!src) {
        for (int q = 0; q < h->nf; ++q) u.w[u.count][q] = h->dirichlet[d][s][q];
        u.count++;
        continue;
      }
      const long long n = h->N / h->n[d];
      const long long blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
      reduce_wavespeed_kernel<<<(int)blocks, 256, 0, st>>>(src, n, h->ndim, h->eos, h->ctl, 0);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess && u.count) {
    bc_wavespeed_kernel<<<1, 32, 0, st>>>(u, h->ndim, h->eos, h->ctl);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->ctl->smax_bc, h->ctl->smax[0], sizeof(h->ctl->smax_bc), cudaMemcpyDeviceToDevice, st);
  return cuda_status(e);
}

// Status of a synchronising call: waits for the handle's stream, then
// compares the device counters with their snapshot from the call's
// launch_init (WCNS_E_NONFINITE, WCNS_E_INADMISSIBLE or WCNS_OK).  The
// step control is returned in *c.
int read_status(wcns_handle *h, StepCtl *c) {
  DevStats s;
  CK(cudaMemcpyAsync(c, h->ctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(&s, h->stats, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return status_from_counts(*c, s, WCNS_OK, WCNS_E_NONFINITE, WCNS_E_INADMISSIBLE);
}

// nsteps SSPRK3 steps.  With graphs enabled (and no per-kernel timing) one
// step is captured once on the private stream and replayed there, ordered
// after the caller's pending work by events; otherwise the kernels are
// launched directly on the caller's stream.
int run_steps(wcns_handle *h, double *W, int nsteps, double dt_fixed, double cfl) {
  if (nsteps <= 0) return WCNS_OK;
  if (!h->use_graphs || h->prof_cap > 0 || !h->cap) {
    for (int k = 0; k < nsteps; ++k) {
      int st = enqueue_step(h, W, dt_fixed, cfl);
      if (st) return st;
    }
    return WCNS_OK;
  }
  if (cudaEventRecord(h->ev_in, h->stream) != cudaSuccess) return WCNS_E_CUDA;
  if (cudaStreamWaitEvent(h->cap, h->ev_in, 0) != cudaSuccess) return WCNS_E_CUDA;
  if (!h->graph || h->graph_W != W || h->graph_dt != dt_fixed || h->graph_cfl != cfl ||
      h->graph_t1 != h->trace_W1 || h->graph_t2 != h->trace_W2) {
    drop_graph(h);
    cudaGraph_t g;
    h->launch_stream = h->cap;
    if (cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      h->launch_stream = h->stream;
      return WCNS_E_CUDA;
    }
    const long long before = h->launches;
    int st = enqueue_step(h, W, dt_fixed, cfl);
    h->launches = before;  // counted when replayed
    cudaError_t e = cudaStreamEndCapture(h->cap, &g);
    h->launch_stream = h->stream;
    if (e == cudaSuccess && st) cudaGraphDestroy(g);  // a partial capture is never launched
    if (st || e != cudaSuccess) return st ? st : WCNS_E_CUDA;
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      h->graph = NULL;
      return WCNS_E_CUDA;
    }
    h->graph_W = W;
    h->graph_dt = dt_fixed;
    h->graph_cfl = cfl;
    h->graph_t1 = h->trace_W1;
    h->graph_t2 = h->trace_W2;
  }
  for (int k = 0; k < nsteps; ++k) {
    if (cudaGraphLaunch(h->graph, h->cap) != cudaSuccess) return WCNS_E_CUDA;
    h->launches += 1 + 3 * h->ndim;
  }
  if (cudaEventRecord(h->ev_out, h->cap) != cudaSuccess) return WCNS_E_CUDA;
  if (cudaStreamWaitEvent(h->stream, h->ev_out, 0) != cudaSuccess) return WCNS_E_CUDA;
  return WCNS_OK;
}

bool valid_bc(int k) { return k >= 0 && k <= 3; }

}  // namespace

extern "C" {

void wcns_default_options(wcns_options *o) {
  if (!o) return;
  o->precision = WCNS_FP64;
  o->scheme = WCNS_SCHEME_PP_WCNS_IS;
  o->eps_is = 1e-40;
  o->eps_ar = 1e-10;
  o->eps_a = 1e-10;
  o->eps_rc = 1e-8;
  o->hs_ar = 1e-11;
  o->hs_a = 1e-11;
  o->hs_rc = 1e-9;
  o->stream = NULL;
}

int wcns_create(const wcns_grid *g, const wcns_bcs *bcs, double gamma_g, double gamma_l, double pinf_l,
                wcns_handle **out) {
  if (!out) return WCNS_E_INVALID_ARG;
  *out = NULL;
  if (!g || !bcs) return WCNS_E_INVALID_ARG;
  if (g->ndim < 1 || g->ndim > 3) return WCNS_E_INVALID_ARG;
  if (!(gamma_g > 1.0) || !(gamma_l > 1.0) || !(pinf_l >= 0.0) || !(gamma_g <= gamma_l) ||
      !isfinite(gamma_g) || !isfinite(gamma_l) || !isfinite(pinf_l))
    return WCNS_E_INVALID_ARG;
  long long N = 1;
  for (int d = 0; d < g->ndim; ++d) {
    if (g->n[d] < 1 || !(g->hi[d] > g->lo[d]) || !isfinite(g->hi[d] - g->lo[d])) return WCNS_E_INVALID_ARG;
    for (int s = 0; s < 2; ++s)
      if (!valid_bc(bcs->kind[d][s])) return WCNS_E_INVALID_ARG;
    if ((bcs->kind[d][0] == WCNS_BC_PERIODIC) != (bcs->kind[d][1] == WCNS_BC_PERIODIC))
      return WCNS_E_INVALID_ARG;
    if ((bcs->kind[d][0] == WCNS_BC_SYMMETRY || bcs->kind[d][1] == WCNS_BC_SYMMETRY) && g->n[d] < 3)
      return WCNS_E_INVALID_ARG;
    // at most 2^30 cells an axis and 2^40 in all, checked before the
    // product is formed so that it cannot overflow
    if (g->n[d] > (1 << 30) || N > (1ll << 40) / g->n[d]) return WCNS_E_INVALID_ARG;
    N *= g->n[d];
  }
  // launch-grid limits of the sweeps (gridDim.y / gridDim.z <= 65535)
  {
    const long long ny = g->ndim > 1 ? g->n[1] : 1, nz = g->ndim > 2 ? g->n[2] : 1;
    // x sweeps: 2 lines a block; y/z sweeps: 8 (mixed) or 16 (FP64) x-columns a block
    if ((ny + 1) / 2 > 65535 || nz > 65535 || (g->ndim > 2 && ny > 65535) ||
        (g->ndim > 1 && ((long long)g->n[0] + 7) / 8 > 65535))
      return WCNS_E_INVALID_ARG;
  }
  wcns_handle *h = (wcns_handle *)calloc(1, sizeof(wcns_handle));
  if (!h) return WCNS_E_CUDA;
  h->ndim = g->ndim;
  h->nf = g->ndim + 4;
  h->N = N;
  for (int d = 0; d < 3; ++d) {
    h->n[d] = d < g->ndim ? g->n[d] : 1;
    h->dx[d] = d < g->ndim ? (g->hi[d] - g->lo[d]) / g->n[d] : 1.0;
    h->inv_dx[d] = d < g->ndim ? 1.0 / h->dx[d] : 0.0;
    for (int s = 0; s < 2; ++s) {
      h->bc[d][s] = d < g->ndim ? bcs->kind[d][s] : WCNS_BC_TRANSMISSIVE;
      for (int q = 0; q < 7; ++q) h->dirichlet[d][s][q] = bcs->dirichlet[d][s][q];
    }
  }
  h->eos = make_eos(gamma_g, gamma_l, pinf_l);
  wcns_default_options(&h->opt);
  h->stream = 0;
  const size_t bytes = sizeof(double) * (size_t)h->nf * (size_t)N;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&h->W1, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->W2, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->L, bytes);
  if (e == cudaSuccess && h->ndim > 1) {
    // node cache: [p | 1/rho] doubles, then [c | bits] 32-bit words
    e = cudaMalloc(&h->node_p, (2 * sizeof(double) + 2 * sizeof(float)) * (size_t)N);
    if (e == cudaSuccess) {
      h->node_ir = h->node_p + N;
      h->node_c = (float *)(h->node_ir + N);
      h->node_ok = (unsigned int *)(h->node_c + N);
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&h->ctl, sizeof(StepCtl));
  if (e == cudaSuccess) e = cudaMalloc(&h->stats, sizeof(DevStats));
  if (e == cudaSuccess) e = cudaMemset(h->stats, 0, sizeof(DevStats));
  if (e == cudaSuccess) e = cudaMemset(h->ctl, 0, sizeof(StepCtl));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming);
  h->launch_stream = h->stream;
  h->use_graphs = 1;
  if (e == cudaSuccess && (update_bc_wavespeed(h) != WCNS_OK || cudaStreamSynchronize(h->stream) != cudaSuccess))
    e = cudaErrorUnknown;
  if (e != cudaSuccess) {
    wcns_destroy(h);
    return WCNS_E_CUDA;
  }
  *out = h;
  return WCNS_OK;
}

int wcns_set_options(wcns_handle *h, const wcns_options *o) {
  if (!h || !o) return WCNS_E_INVALID_ARG;
  if (o->precision != WCNS_FP64 && o->precision != WCNS_MIXED) return WCNS_E_INVALID_ARG;
  if (o->scheme < 0 || o->scheme > 2) return WCNS_E_INVALID_ARG;
  if (!valid_tolerances(*o))
    return WCNS_E_INVALID_ARG;
  h->opt = *o;
  h->stream = (cudaStream_t)o->stream;
  h->launch_stream = h->stream;
  drop_graph(h);
  return WCNS_OK;
}

int wcns_get_options(const wcns_handle *h, wcns_options *o) {
  if (!h || !o) return WCNS_E_INVALID_ARG;
  *o = h->opt;
  return WCNS_OK;
}

int wcns_set_dirichlet_face(wcns_handle *h, int axis, int side, const double *W_face) {
  if (!h || axis < 0 || axis >= h->ndim || side < 0 || side > 1) return WCNS_E_INVALID_ARG;
  if (h->bc[axis][side] != WCNS_BC_DIRICHLET) return WCNS_E_INVALID_ARG;
  CK(cudaStreamSynchronize(h->stream));
  if (h->cap) CK(cudaStreamSynchronize(h->cap));
  const size_t bytes = sizeof(double) * (size_t)h->nf * (size_t)(h->N / h->n[axis]);
  if (!W_face) {
    if (h->dir_face[axis][side]) {
      drop_graph(h);  // the captured launches carry the buffer's address
      CK(cudaFree(h->dir_face[axis][side]));
      h->dir_face[axis][side] = NULL;
    }
    return update_bc_wavespeed(h);
  }
  if (!h->dir_face[axis][side]) {
    drop_graph(h);
    CK(cudaMalloc(&h->dir_face[axis][side], bytes));
  }
  CK(cudaMemcpy(h->dir_face[axis][side], W_face, bytes, cudaMemcpyHostToDevice));
  return update_bc_wavespeed(h);
}

int wcns_set_stage_trace(wcns_handle *h, double *W1_out, double *W2_out) {
  if (!h || (!W1_out) != (!W2_out)) return WCNS_E_INVALID_ARG;
  h->trace_W1 = W1_out;
  h->trace_W2 = W2_out;
  return WCNS_OK;
}

int wcns_rhs(wcns_handle *h, const double *W, double *dWdt, double dt) {
  if (!h || !W || !dWdt || !(dt >= 0.0) || !isfinite(dt)) return WCNS_E_INVALID_ARG;
  const size_t bytes = sizeof(double) * (size_t)h->nf * (size_t)h->N;
  if ((const char *)W < (const char *)dWdt + bytes && (const char *)dWdt < (const char *)W + bytes)
    return WCNS_E_INVALID_ARG;
  int st = launch_init(h, 0.0, INFINITY);
  if (!st && h->ndim > 1) st = launch_reduce(h, W, 3);
  if (!st) st = launch_begin(h, dt > 0.0 ? dt : 1e-300, 0.0, 0);
  if (!st) st = enqueue_rhs(h, W, dWdt);
  return st;
}

int wcns_max_wavespeed(wcns_handle *h, const double *W, double out[3]) {
  if (!h || !W || !out) return WCNS_E_INVALID_ARG;
  int st = launch_init(h, 0.0, INFINITY);
  if (!st) st = launch_reduce(h, W, 3);
  if (st) return st;
  StepCtl c;
  CK(cudaMemcpyAsync(&c, h->ctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (int d = 0; d < 3; ++d) {
    unsigned long long b = c.smax[3][d];
    double v;
    memcpy(&v, &b, sizeof(v));
    out[d] = d < h->ndim ? v : 0.0;
  }
  return WCNS_OK;
}

int wcns_rk3_step(wcns_handle *h, double *W, double dt) {
  if (!h || !W || !(dt > 0.0) || !isfinite(dt)) return WCNS_E_INVALID_ARG;
  int st = launch_init(h, 0.0, INFINITY);
  if (!st && h->ndim > 1) st = launch_reduce(h, W, 3);
  if (!st) st = enqueue_step(h, W, dt, 0.0);  // dt varies per call: direct launches
  return st;
}

int wcns_advance_steps(wcns_handle *h, double *W, int nsteps, double cfl, double dt_fixed, double *t_io) {
  if (!h || !W || nsteps < 0 || !(dt_fixed >= 0.0) || !isfinite(dt_fixed)) return WCNS_E_INVALID_ARG;
  if (dt_fixed == 0.0 && !(cfl > 0.0 && cfl <= 1.0)) return WCNS_E_INVALID_ARG;
  const double t0 = t_io ? *t_io : 0.0;
  int st = launch_init(h, t0, INFINITY);
  if (!st && (h->ndim > 1 || dt_fixed == 0.0)) st = launch_reduce(h, W, 3);
  if (!st) st = run_steps(h, W, nsteps, dt_fixed, cfl);
  if (st) return st;
  StepCtl c;
  st = read_status(h, &c);
  if (t_io) *t_io = c.t;
  return st;
}

int wcns_advance_to(wcns_handle *h, double *W, double t0, double t_end, double cfl, double *t_out,
                    long *steps_out) {
  if (!h || !W || !isfinite(t0) || !isfinite(t_end) || !(cfl > 0.0 && cfl <= 1.0)) return WCNS_E_INVALID_ARG;
  int st = launch_init(h, t0, t_end);
  if (!st) st = launch_reduce(h, W, 3);
  if (st) return st;
  StepCtl c;
  int batch = 8;
  for (;;) {
    st = run_steps(h, W, batch, 0.0, cfl);
    if (st) return st;
    st = read_status(h, &c);
    if (t_out) *t_out = c.t;
    if (steps_out) *steps_out = (long)c.steps;
    // a non-finite wave speed makes dt and t NaN: report it before the
    // t < t_end test (false for NaN) could end the loop as if t_end was reached
    if (!isfinite(c.t) || !isfinite(c.dt) || (c.active && c.dt <= 0.0)) return WCNS_E_NONFINITE;
    if (st) return st;  // a non-finite update or an inadmissible stage input
    if (!c.active || !(c.t < t_end)) break;
    if (batch < 256) batch *= 2;
  }
  return WCNS_OK;
}

int wcns_advance_steps_host(wcns_handle *h, double *W_host, int nsteps, double cfl, double dt_fixed,
                            double *t_io) {
  if (!h || !W_host) return WCNS_E_INVALID_ARG;
  const size_t bytes = sizeof(double) * (size_t)h->nf * (size_t)h->N;
  if (!h->Wh) CK(cudaMalloc(&h->Wh, bytes));
  CK(cudaMemcpyAsync(h->Wh, W_host, bytes, cudaMemcpyHostToDevice, h->stream));
  double t = t_io ? *t_io : 0.0;
  const int st = wcns_advance_steps(h, h->Wh, nsteps, cfl, dt_fixed, &t);
  // the state comes back also when the steps report a non-finite or
  // inadmissible state (the caller sees what the device holds)
  if (st != WCNS_OK && st != WCNS_E_NONFINITE && st != WCNS_E_INADMISSIBLE) return st;
  CK(cudaMemcpyAsync(W_host, h->Wh, bytes, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (t_io) *t_io = t;
  return st;
}

int wcns_get_stats(wcns_handle *h, wcns_stats *out) {
  if (!h || !out) return WCNS_E_INVALID_ARG;
  DevStats s;
  CK(cudaMemcpyAsync(&s, h->stats, sizeof(s), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  out->interp_limited = (long long)s.interp_limited;
  out->interp_hard = (long long)s.interp_hard;
  out->flux_limited = (long long)s.flux_limited;
  out->flux_hard = (long long)s.flux_hard;
  out->nonfinite = (long long)s.nonfinite;
  out->inadmissible = (long long)s.inadmissible;
  out->midpoints = (long long)s.midpoints;
  out->fp64_fallbacks = (long long)s.fp64_fallbacks;
  return WCNS_OK;
}

int wcns_reset_stats(wcns_handle *h) {
  if (!h) return WCNS_E_INVALID_ARG;
  CK(cudaMemsetAsync(h->stats, 0, sizeof(DevStats), h->stream));
  return WCNS_OK;
}

int wcns_profile_enable(wcns_handle *h, int capacity) {
  if (!h || capacity < 0) return WCNS_E_INVALID_ARG;
  // the timing events are re-created: let every launch that records one finish
  CK(cudaStreamSynchronize(h->stream));
  if (h->cap) CK(cudaStreamSynchronize(h->cap));
  profile_free(h);
  if (capacity == 0) return WCNS_OK;
  h->prof_ev = (cudaEvent_t *)calloc(2 * (size_t)capacity, sizeof(cudaEvent_t));
  h->prof_dir = (int *)calloc((size_t)capacity, sizeof(int));
  if (!h->prof_ev || !h->prof_dir) {
    free(h->prof_ev);
    free(h->prof_dir);
    h->prof_ev = NULL;
    h->prof_dir = NULL;
    return WCNS_E_INVALID_ARG;
  }
  for (int k = 0; k < 2 * capacity; ++k) {
    if (cudaEventCreate(&h->prof_ev[k]) != cudaSuccess) {
      h->prof_cap = k / 2;
      profile_free(h);
      return WCNS_E_CUDA;
    }
  }
  h->prof_cap = capacity;
  return WCNS_OK;
}

int wcns_profile_read(wcns_handle *h, wcns_profile *out) {
  if (!h || !out) return WCNS_E_INVALID_ARG;
  memset(out, 0, sizeof(*out));
  CK(cudaStreamSynchronize(h->stream));
  for (int k = 0; k < h->prof_n; ++k) {
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, h->prof_ev[2 * k], h->prof_ev[2 * k + 1]));
    out->launches[h->prof_dir[k]] += 1;
    out->ms[h->prof_dir[k]] += ms;
  }
  out->dropped = h->prof_dropped;
  h->prof_n = 0;
  h->prof_dropped = 0;
  return WCNS_OK;
}

int wcns_nfields(const wcns_handle *h) { return h ? h->nf : 0; }
long long wcns_ncells(const wcns_handle *h) { return h ? h->N : 0; }
long long wcns_launch_count(const wcns_handle *h) { return h ? h->launches : 0; }

const char *wcns_strerror(int s) {
  switch (s) {
    case WCNS_OK: return "ok";
    case WCNS_E_INVALID_ARG: return "invalid argument";
    case WCNS_E_CUDA: return "CUDA runtime error";
    case WCNS_E_INADMISSIBLE: return "input state outside the admissible set";
    case WCNS_E_NONFINITE: return "non-finite value";
    case WCNS_E_UNSUPPORTED: return "unsupported option combination";
    case WCNS_E_TOO_LARGE:
      return "problem too large for the fixed no-allocation scratch (needs 3 * nf * ncells <= "
             "WCNS_NOALLOC_MAX_DOUBLES doubles)";
    default: return "unknown status";
  }
}

void wcns_destroy(wcns_handle *h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  if (h->cap) cudaStreamSynchronize(h->cap);
  drop_graph(h);
  if (h->ev_in) cudaEventDestroy(h->ev_in);
  if (h->ev_out) cudaEventDestroy(h->ev_out);
  if (h->cap) cudaStreamDestroy(h->cap);
  h->ev_in = h->ev_out = NULL;
  h->cap = NULL;
  for (int d = 0; d < 3; ++d)
    for (int s2 = 0; s2 < 2; ++s2) cudaFree(h->dir_face[d][s2]);
  profile_free(h);
  cudaFree(h->W1);
  cudaFree(h->W2);
  cudaFree(h->L);
  cudaFree(h->node_p);
  cudaFree(h->Wh);
  cudaFree(h->ctl);
  cudaFree(h->stats);
  free(h);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free SSPRK3 step.  Its scratch is one file-scope device array:
//   [ W1 | W2 | L ]  (3 * nf * ncells doubles), in 2D/3D then the node cache
//   (3 * ncells doubles), and StepCtl, DevStats
// in a separate small region.  Host code must not pass the array's name to
// a kernel (in host code it is a host-side stand-in, not a device address):
// its device address is looked up once per device with cudaGetSymbolAddress.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {
static __device__ __align__(256) double g_noalloc_states[WCNS_NOALLOC_MAX_DOUBLES];
static __device__ __align__(256) unsigned char g_noalloc_ctl[1024];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_states_ptr[kMaxDevices];
unsigned char *g_noalloc_ctl_ptr[kMaxDevices];

// Once per device, with that device current.
int noalloc_setup(int dev, double **states, unsigned char **ctl) {
  if (dev < 0 || dev >= kMaxDevices) return WCNS_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_states_ptr[dev]) {
    void *p = NULL, *q = NULL;
    if (cudaGetSymbolAddress(&p, g_noalloc_states) != cudaSuccess) return WCNS_E_CUDA;
    if (cudaGetSymbolAddress(&q, g_noalloc_ctl) != cudaSuccess) return WCNS_E_CUDA;
    g_noalloc_states_ptr[dev] = (double *)p;
    g_noalloc_ctl_ptr[dev] = (unsigned char *)q;
  }
  *states = g_noalloc_states_ptr[dev];
  *ctl = g_noalloc_ctl_ptr[dev];
  return WCNS_OK;
}
}  // namespace

extern "C" int wcns_rk3_step_noalloc(const wcns_grid *g, const wcns_bcs *bcs, double gamma_g, double gamma_l,
                                     double pinf_l, const wcns_options *opt, double *W, double dt) {
  if (!g || !bcs || !W || !(dt > 0.0) || !isfinite(dt)) return WCNS_E_INVALID_ARG;
  // Same validation as wcns_create, on a handle that lives on the stack.
  if (g->ndim < 1 || g->ndim > 3) return WCNS_E_INVALID_ARG;
  if (!(gamma_g > 1.0) || !(gamma_l > 1.0) || !(pinf_l >= 0.0) || !(gamma_g <= gamma_l) ||
      !isfinite(gamma_g) || !isfinite(gamma_l) || !isfinite(pinf_l))
    return WCNS_E_INVALID_ARG;
  long long N = 1;
  for (int d = 0; d < g->ndim; ++d) {
    if (g->n[d] < 1 || !(g->hi[d] > g->lo[d]) || !isfinite(g->hi[d] - g->lo[d])) return WCNS_E_INVALID_ARG;
    for (int s2 = 0; s2 < 2; ++s2)
      if (!valid_bc(bcs->kind[d][s2])) return WCNS_E_INVALID_ARG;
    if ((bcs->kind[d][0] == WCNS_BC_PERIODIC) != (bcs->kind[d][1] == WCNS_BC_PERIODIC)) return WCNS_E_INVALID_ARG;
    if ((bcs->kind[d][0] == WCNS_BC_SYMMETRY || bcs->kind[d][1] == WCNS_BC_SYMMETRY) && g->n[d] < 3)
      return WCNS_E_INVALID_ARG;
    if (g->n[d] > (1 << 30) || N > (1ll << 40) / g->n[d]) return WCNS_E_TOO_LARGE;
    N *= g->n[d];
  }
  {
    const long long ny = g->ndim > 1 ? g->n[1] : 1, nz = g->ndim > 2 ? g->n[2] : 1;
    if ((ny + 1) / 2 > 65535 || nz > 65535 || (g->ndim > 2 && ny > 65535) ||
        (g->ndim > 1 && ((long long)g->n[0] + 7) / 8 > 65535))
      return WCNS_E_INVALID_ARG;
  }
  const int nf = g->ndim + 4;
  // three states, plus the mixed sweeps' node cache in 2D/3D (3 doubles a cell)
  if ((3ll * nf + (g->ndim > 1 ? 3 : 0)) * N > WCNS_NOALLOC_MAX_DOUBLES) return WCNS_E_TOO_LARGE;
  wcns_options o;
  wcns_default_options(&o);
  if (opt) o = *opt;
  if (o.precision != WCNS_FP64 && o.precision != WCNS_MIXED) return WCNS_E_INVALID_ARG;
  if (o.scheme < 0 || o.scheme > 2) return WCNS_E_INVALID_ARG;
  if (!valid_tolerances(o)) return WCNS_E_INVALID_ARG;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return WCNS_E_CUDA;
  double *states = NULL;
  unsigned char *ctlmem = NULL;
  int st = noalloc_setup(dev, &states, &ctlmem);
  if (st) return st;

  wcns_handle h;
  memset(&h, 0, sizeof(h));
  h.ndim = g->ndim;
  h.nf = nf;
  h.N = N;
  for (int d = 0; d < 3; ++d) {
    h.n[d] = d < g->ndim ? g->n[d] : 1;
    h.dx[d] = d < g->ndim ? (g->hi[d] - g->lo[d]) / g->n[d] : 1.0;
    h.inv_dx[d] = d < g->ndim ? 1.0 / h.dx[d] : 0.0;
    for (int s2 = 0; s2 < 2; ++s2) {
      h.bc[d][s2] = d < g->ndim ? bcs->kind[d][s2] : WCNS_BC_TRANSMISSIVE;
      for (int q = 0; q < 7; ++q) h.dirichlet[d][s2][q] = bcs->dirichlet[d][s2][q];
    }
  }
  h.eos = make_eos(gamma_g, gamma_l, pinf_l);
  h.opt = o;
  h.stream = (cudaStream_t)o.stream;
  h.launch_stream = h.stream;
  const size_t M = (size_t)nf * (size_t)N;
  h.W1 = states;
  h.W2 = states + M;
  h.L = states + 2 * M;
  if (h.ndim > 1) {  // node cache, laid out as in wcns_create
    h.node_p = states + 3 * M;
    h.node_ir = h.node_p + N;
    h.node_c = (float *)(h.node_ir + N);
    h.node_ok = (unsigned int *)(h.node_c + N);
  }
  // small region: StepCtl | DevStats (the uniform Dirichlet states reach
  // the device as kernel arguments, from this stack frame's handle)
  constexpr size_t kStatsOff = ((sizeof(StepCtl) + 15) / 16) * 16;
  static_assert(kStatsOff + sizeof(DevStats) <= sizeof(g_noalloc_ctl), "no-alloc control region too small");
  h.ctl = (StepCtl *)ctlmem;
  h.stats = (DevStats *)(ctlmem + kStatsOff);
  // The counters keep the previous call's values: clear them.
  if (cudaMemsetAsync(h.stats, 0, sizeof(DevStats), h.stream) != cudaSuccess) return WCNS_E_CUDA;
  st = update_bc_wavespeed(&h);
  if (!st) st = launch_init(&h, 0.0, INFINITY);
  if (!st && h.ndim > 1) st = launch_reduce(&h, W, 3);
  if (!st) st = enqueue_step(&h, W, dt, 0.0);
  return st;
}
