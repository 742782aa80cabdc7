// Batched mode of the C ABI: many independent 1D or 2D problems of uneven
// sizes advanced together.  In 1D every SSPRK3 stage is ONE persistent
// launch over a work list of (problem, tile) pairs; in 2D one persistent
// launch per direction (the first writes the flux differences, the second
// adds its own and combines the stage).  Each problem keeps its own CFL time
// step and directional split (Sec. 3.3: dt_k = cfl / sum_d max(|u_d| + c)/dx_d,
// lambda_d from the stage input's maxima); a whole step (dt update + every
// stage) is captured once into a CUDA graph and replayed.  The tile length
// (1D) and the persistent grid's blocks per SM are chosen by a small
// autotuner on the first advance.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <type_traits>
#include <vector>

#include "../../include/wcns.h"
#include "wcns_mixed_body.cuh"

using namespace wcns;

// Mixed batch tiles: the single-pass midpoint loop (false) or the fast pass
// with certification failures deferred to a second pass (true).
#ifndef BATCH_MIXED_DEFER
#define BATCH_MIXED_DEFER false
#endif

namespace {

struct BatchArgs {
  const long long *offsets;   // first cell of each problem in the packed array
  const int *ncell;           // cells per problem
  const double *inv_dx;       // 1/dx per problem
  const double *dt;           // current step size per problem
  unsigned long long *smax;   // max(|u|+c) bits of each problem's newest state
  const int *tile_prob;       // problem of each tile
  const int *tile_first;      // first midpoint of each tile
  int ntiles;
};

// Geometry policy: one tile of one problem (a single 1D line).
template <class T>
struct BatchGeo {
  const BatchArgs &b;
  int prob, tile0, n;
  long long base;
  __device__ BatchGeo(const BatchArgs &b_, int t) : b(b_) {
    prob = b.tile_prob[t];
    tile0 = b.tile_first[t];
    base = b.offsets[prob];
    n = b.ncell[prob];
  }
  __device__ Line line(int) const {
    Line r;
    r.base = base;
    r.face = 0;
    r.stride = 1;
    r.n = n;
    r.valid = true;
    return r;
  }
  __device__ double dt() const { return b.dt[prob]; }
  __device__ double inv_dx() const { return b.inv_dx[prob]; }
  __device__ double lam() const { return b.dt[prob] * b.inv_dx[prob]; }  // 1D: sigma = 1
  __device__ unsigned long long *smax_slot(int) const { return &b.smax[prob]; }
  __device__ double l_unit() const { return 1.0; }       // 1D: L is never read
  __device__ double accum_scale() const { return 1.0; }  // 1D: no accumulating sweep
};

// MIXED selects the mixed-precision body (wcns_mixed_body.cuh).  Mixed
// tiles target BATCH_MIXED_WARPS resident warps per SM (a register cap of
// 65536 / (32 BATCH_MIXED_WARPS) per thread); the FP64 body keeps its
// registers.  On the 4096-problem batch 32 warps (64 registers, more
// spills) beat 28, 24, 20 and 16: the single-pass body is latency bound.
#ifndef BATCH_MIXED_WARPS
#define BATCH_MIXED_WARPS 32
#endif
template <bool MIXED, class T>
__global__ void __launch_bounds__(T::THREADS, MIXED ? BATCH_MIXED_WARPS * 32 / T::THREADS : 1)
    batch_sweep_kernel(const SweepArgs a, const BatchArgs b) {
  extern __shared__ double smem_raw[];
  for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
    if constexpr (MIXED)
      sweep_body_mixed<1, 0, T, BATCH_MIXED_DEFER>(a, BatchGeo<T>(b, t), smem_raw);
    else
      sweep_body<1, 0, double, T>(a, BatchGeo<T>(b, t), smem_raw);
    __syncthreads();
  }
}

template <bool MIXED, class T>
constexpr size_t batch_smem() {
  return MIXED ? SmemMixed<1, T>::BYTES : Smem<1, 0, T>::BYTES;
}

// max(|u| + c) per problem (FP64 EOS, Sec. 2, with the single-grid
// reduction's formula), one block per tile.
__global__ void batch_reduce_kernel(const double *__restrict__ W, long long total, EosConst e, BatchArgs b,
                                    int tile_cells) {
  for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
    const int prob = b.tile_prob[t];
    const int first = b.tile_first[t];
    const int n = b.ncell[prob];
    double smax = 0.0;
    for (int i = first + threadIdx.x; i < min(first + tile_cells, n); i += blockDim.x) {
      const long long idx = b.offsets[prob] + i;
      const double m = W[2 * total + idx];
      double s;
      state_wavespeeds(W[idx], W[total + idx], &m, W[3 * total + idx], W[4 * total + idx], 1, e, &s);
      smax = (s > smax || s != s) ? s : smax;
    }
    unsigned long long bits = __double_as_longlong(smax);
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
      bits = ob > bits ? ob : bits;
    }
    if ((threadIdx.x & 31) == 0 && bits) atomicMax(&b.smax[prob], bits);
  }
}

// Start of a step for every problem: dt_k from the newest max(|u|+c), then
// clear the accumulator that the step's last stage refills.
__global__ void batch_begin_kernel(int nprob, const double *inv_dx, double *dt, unsigned long long *smax,
                                   double cfl, double *t_acc) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nprob) return;
  const double s = __longlong_as_double(smax[k]);
  const double d = cfl / (s * inv_dx[k]);
  dt[k] = d;
  smax[k] = 0ull;
  if (t_acc) t_acc[k] += d;
}

// ---------------------------------------------------------------------------
// 2D batches.  Problem k is an nx_k x ny_k grid stored row-major (x fastest)
// in columns offsets[k] .. offsets[k] + nx_k ny_k - 1 of the packed
// [6][total] state.  Per problem the tables hold what a single grid keeps in
// its step control: dt, the wave-speed maxima of the four stage states
// (smax[k][0..3][d], FP64 bit patterns, as StepCtl::smax) and, for the mixed
// sweeps, the scaling of the L array.
// ---------------------------------------------------------------------------
struct Batch2Args {
  const long long *offsets;
  const int *nx, *ny;
  const double *inv_dx;        // [nprob][2]: 1/dx, 1/dy
  const double *dt;            // [nprob]
  unsigned long long *smax;    // [nprob][4][2]
  const double *l_unit;        // [nprob]: 1/dx of the first mixed sweep (combine scale)
  const int *tile_prob, *tile_first, *tile_line;  // work list of this direction
  int ntiles;
};

// Geometry policy: one (problem, tile) of a 2D batch; lines are rows (DIR
// 0) or columns (DIR 1) of the problem's grid, as in GridGeo.
template <int DIR, class T>
struct Batch2Geo {
  const SweepArgs &a;
  const Batch2Args &b;
  int prob, tile0, line0, nx, ny;
  long long off;
  __device__ Batch2Geo(const SweepArgs &a_, const Batch2Args &b_, int t) : a(a_), b(b_) {
    prob = b.tile_prob[t];
    tile0 = b.tile_first[t];
    line0 = b.tile_line[t];
    nx = b.nx[prob];
    ny = b.ny[prob];
    off = b.offsets[prob];
  }
  __device__ Line line(int l) const {
    Line r;
    if (DIR == 0) {
      int y = line0 + l;
      r.valid = y < ny;
      y = min(y, ny - 1);
      r.face = y;
      r.base = off + (long long)y * nx;
      r.stride = 1;
      r.n = nx;
    } else {
      int x = line0 + l;
      r.valid = x < nx;
      x = min(x, nx - 1);
      r.face = x;
      r.base = off + x;
      r.stride = nx;
      r.n = ny;
    }
    return r;
  }
  __device__ double dt() const { return b.dt[prob]; }
  __device__ double inv_dx() const { return b.inv_dx[2 * prob + DIR]; }
  // lambda_d = dt sum_j tau_j / max(|u_d| + c), tau_j = max(|u_j| + c)/dx_j
  // of the stage input (Sec. 3.3), in GridGeo::lam's order of operations
  __device__ double lam() const {
    const unsigned long long *sm = b.smax + (size_t)(4 * prob + a.stage) * 2;
    double tsum = 0.0;
#pragma unroll
    for (int j = 0; j < 2; ++j) tsum += __longlong_as_double(sm[j]) * b.inv_dx[2 * prob + j];
    return b.dt[prob] * tsum / __longlong_as_double(sm[DIR]);
  }
  __device__ unsigned long long *smax_slot(int j) const {
    return &b.smax[(size_t)(4 * prob + a.stage + 1) * 2 + j];
  }
  __device__ double l_unit() const { return b.l_unit[prob]; }
  __device__ double accum_scale() const { return 1.0; }  // 2D: no accumulating sweep
};

// One direction of one stage of every problem: a persistent loop over the
// direction's work list.
template <bool MIXED, int DIR, class T>
__global__ void __launch_bounds__(T::THREADS, MIXED ? 3 : 1)
    batch2_sweep_kernel(const SweepArgs a, const Batch2Args b) {
  extern __shared__ double smem_raw[];
  for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
    if constexpr (MIXED)
      sweep_body_mixed<2, DIR, T>(a, Batch2Geo<DIR, T>(a, b, t), smem_raw);
    else
      sweep_body<2, DIR, double, T>(a, Batch2Geo<DIR, T>(a, b, t), smem_raw);
    __syncthreads();
  }
}

// Tiles of the 2D batch (both precisions): x tiles of 4 rows x 58 cells and
// y tiles of 8 columns x 26 cells, 256 nodes each (one node per thread),
// shaped for problems of tens to hundreds of cells an axis.
using Batch2TileX = TileT<4, 59, 256>;
using Batch2TileY = TileT<8, 27, 256>;

template <bool MIXED, int DIR>
constexpr size_t batch2_smem() {
  using T = typename std::conditional<DIR == 0, Batch2TileX, Batch2TileY>::type;
  return MIXED ? SmemMixed<2, T>::BYTES : Smem<2, DIR, T>::BYTES;
}

template <bool MIXED, int DIR>
cudaError_t launch_batch2(const SweepArgs &a, const Batch2Args &b, int grid, cudaStream_t s) {
  using T = typename std::conditional<DIR == 0, Batch2TileX, Batch2TileY>::type;
  const size_t bytes = batch2_smem<MIXED, DIR>();
  static std::atomic<unsigned long long> configured{0};
  cudaError_t e = configure_once(configured, [&] {
    return cudaFuncSetAttribute(batch2_sweep_kernel<MIXED, DIR, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes);
  });
  if (e != cudaSuccess) return e;
  batch2_sweep_kernel<MIXED, DIR, T><<<grid, T::THREADS, bytes, s>>>(a, b);
  return cudaGetLastError();
}

template <bool MIXED, int DIR>
int batch2_max_blocks_per_sm() {
  using T = typename std::conditional<DIR == 0, Batch2TileX, Batch2TileY>::type;
  int nb = 0;
  const size_t bytes = batch2_smem<MIXED, DIR>();
  cudaFuncSetAttribute(batch2_sweep_kernel<MIXED, DIR, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch2_sweep_kernel<MIXED, DIR, T>, T::THREADS, bytes) !=
      cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

// max(|u_d| + c) of every cell of every problem (FP64, the single-grid
// reduction's formula) into smax[k][3][d]; one block per x-sweep tile.
__global__ void batch2_reduce_kernel(const double *__restrict__ W, long long total, EosConst e, Batch2Args b) {
  using T = Batch2TileX;
  for (int t = blockIdx.x; t < b.ntiles; t += gridDim.x) {
    const int prob = b.tile_prob[t];
    const int nx = b.nx[prob], ny = b.ny[prob];
    double smax[2] = {0.0, 0.0};
    for (int q = threadIdx.x; q < T::TL * (T::TM - 1); q += blockDim.x) {
      const int y = b.tile_line[t] + q / (T::TM - 1);
      const int x = b.tile_first[t] + q % (T::TM - 1);
      if (y >= ny || x >= nx) continue;
      const long long idx = b.offsets[prob] + (long long)y * nx + x;
      const double m[2] = {W[2 * total + idx], W[3 * total + idx]};
      double sp[2];
      state_wavespeeds(W[idx], W[total + idx], m, W[4 * total + idx], W[5 * total + idx], 2, e, sp);
      for (int j = 0; j < 2; ++j) smax[j] = (sp[j] > smax[j] || sp[j] != sp[j]) ? sp[j] : smax[j];
    }
    for (int j = 0; j < 2; ++j) {
      unsigned long long bits = __double_as_longlong(smax[j]);
      for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, bits, o);
        bits = ob > bits ? ob : bits;
      }
      if ((threadIdx.x & 31) == 0 && bits) atomicMax(&b.smax[(size_t)(4 * prob + 3) * 2 + j], bits);
    }
  }
}

// Start of a step for every problem (as step_begin_kernel for one grid):
// the maxima of W^n (left in slot 3 by the previous step's combine or by the
// reduction) move to slot 0, dt = cfl / sum_d smax_d / dx_d, the other slots
// are cleared for the stages to refill.
__global__ void batch2_begin_kernel(int nprob, const double *inv_dx, double *dt, unsigned long long *smax,
                                    double cfl, double *t_acc) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nprob) return;
  unsigned long long *sm = smax + (size_t)k * 8;
  double tsum = 0.0;
  for (int d = 0; d < 2; ++d) {
    sm[d] = sm[6 + d];
    tsum += __longlong_as_double(sm[d]) * inv_dx[2 * k + d];
  }
  for (int q = 2; q < 8; ++q) sm[q] = 0ull;
  const double h = cfl / tsum;
  dt[k] = h;
  if (t_acc) t_acc[k] += h;
}

// DevStats counts at the start of a batch advance, for its status.
__global__ void batch_snapshot_kernel(const DevStats *s, StepCtl *c) {
  c->stat0[0] = s->inadmissible;
  c->stat0[1] = s->nonfinite;
}

typedef cudaError_t (*BatchLauncher)(const SweepArgs &, const BatchArgs &, int grid, cudaStream_t);

// A batch tile: TH threads and TH - TRIM midpoints (TH - TRIM + 5 nodes).
// Mixed tiles use TRIM = 5, so that the node stage is exactly one node per
// thread (its FP64 work would otherwise leave most threads waiting at the
// barrier for a few); the FP64 tiles keep TRIM = 0, which measured faster.
template <int TH, int TRIM>
using BatchTile = TileT<1, TH - TRIM, TH>;

template <bool MIXED, int TH, int TRIM>
cudaError_t launch_batch(const SweepArgs &a, const BatchArgs &b, int grid, cudaStream_t s) {
  using T = BatchTile<TH, TRIM>;
  const size_t bytes = batch_smem<MIXED, T>();
  static std::atomic<unsigned long long> configured{0};
  cudaError_t e = configure_once(configured, [&] {
    return cudaFuncSetAttribute(batch_sweep_kernel<MIXED, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)bytes);
  });
  if (e != cudaSuccess) return e;
  batch_sweep_kernel<MIXED, T><<<grid, T::THREADS, bytes, s>>>(a, b);
  return cudaGetLastError();
}

template <bool MIXED, int TH, int TRIM>
int max_blocks_per_sm() {
  using T = BatchTile<TH, TRIM>;
  int nb = 0;
  const size_t bytes = batch_smem<MIXED, T>();
  cudaFuncSetAttribute(batch_sweep_kernel<MIXED, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_sweep_kernel<MIXED, T>, T::THREADS, bytes) !=
      cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

// Tile variants the autotuner chooses from; a variant serves the precision
// whose launcher is set.
struct Variant {
  int tm;  // midpoints per tile (tiles cover tm - 1 cells)
  BatchLauncher fp64, mixed;
  int (*occ64)(), (*occm)();
};
const Variant kVariants[] = {
    {BatchTile<64, 0>::TM, launch_batch<false, 64, 0>, nullptr, max_blocks_per_sm<false, 64, 0>, nullptr},
    {BatchTile<128, 0>::TM, launch_batch<false, 128, 0>, nullptr, max_blocks_per_sm<false, 128, 0>, nullptr},
    {BatchTile<256, 0>::TM, launch_batch<false, 256, 0>, nullptr, max_blocks_per_sm<false, 256, 0>, nullptr},
    {BatchTile<64, 5>::TM, nullptr, launch_batch<true, 64, 5>, nullptr, max_blocks_per_sm<true, 64, 5>},
    {BatchTile<128, 5>::TM, nullptr, launch_batch<true, 128, 5>, nullptr, max_blocks_per_sm<true, 128, 5>},
    {BatchTile<256, 5>::TM, nullptr, launch_batch<true, 256, 5>, nullptr, max_blocks_per_sm<true, 256, 5>},
};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

}  // namespace

struct wcns_batch {
  int ndim;  // 1 or 2
  int nprob;
  long long total;
  EosConst eos;
  int bc_lo, bc_hi;  // 1D
  int bc[2][2];      // 2D: [axis][side]
  wcns_options opt;
  cudaStream_t stream;      // caller's stream
  cudaStream_t cap;         // private stream for graph capture and replay
  cudaEvent_t ev_in, ev_out;
  int sms;
  // device tables
  long long *offsets;
  int *ncell;
  double *inv_dx, *dt;
  unsigned long long *smax, *smax_scratch;
  double *W1, *W2, *Wtrial;
  DevStats *stats;
  StepCtl *ctl;  // counter snapshot of the current advance (stat0); the
                 // batch geometry takes dt from its per-problem tables
  // per tile length: work list
  int *tile_prob[kNumVariants], *tile_first[kNumVariants];
  int ntiles[kNumVariants];
  // autotuned choice
  int tuned, variant, grid;
  // 2D batches: per-problem sizes, 1/dx and 1/dy, stage maxima, L scale;
  // the RHS accumulator and the mixed sweeps' node cache; one work list per
  // direction (problem, first midpoint, first line of each tile)
  int *nx2, *ny2;
  double *inv_dx2, *l_unit2, *L2;
  unsigned long long *smax2;
  double *node_p, *node_ir;
  float *node_c;
  unsigned int *node_ok;
  int *tl_prob[2], *tl_first[2], *tl_line[2];
  int ntl[2];
  // captured step
  cudaGraphExec_t graph;
  double *graph_W;
  double graph_cfl;
  double *graph_t;
  long long launches;
};

namespace {

BatchArgs batch_args(wcns_batch *b, int v, unsigned long long *smax_out) {
  BatchArgs a;
  a.offsets = b->offsets;
  a.ncell = b->ncell;
  a.inv_dx = b->inv_dx;
  a.dt = b->dt;
  a.smax = smax_out;
  a.tile_prob = b->tile_prob[v];
  a.tile_first = b->tile_first[v];
  a.ntiles = b->ntiles[v];
  return a;
}

SweepArgs stage_args(wcns_batch *b, int s, const double *Win, double *Wout, const double *Wn) {
  SweepArgs a;
  memset(&a, 0, sizeof(a));
  a.n[0] = 1;
  a.n[1] = a.n[2] = 1;
  a.ncell = b->total;
  a.bc_lo = b->bc_lo;
  a.bc_hi = b->bc_hi;
  a.eos = b->eos;
  a.tol.eps_ar = b->opt.eps_ar;
  a.tol.eps_a = b->opt.eps_a;
  a.tol.eps_rc = b->opt.eps_rc;
  a.tol.hs_ar = b->opt.hs_ar;
  a.tol.hs_a = b->opt.hs_a;
  a.tol.hs_rc = b->opt.hs_rc;
  set_cert(a.tol);
  a.eps_is = b->opt.eps_is;
  a.eps_is32 = (float)fmax(b->opt.eps_is, 1e-30);
  a.scheme = b->opt.scheme;
  a.epilogue = EPI_COMBINE;
  a.read_L = 0;
  const double ra[3] = {0.0, 0.75, 1.0 / 3.0};
  const double rb[3] = {1.0, 0.25, 2.0 / 3.0};
  a.rk_a = ra[s];
  a.rk_b = rb[s];
  a.stage = s;
  a.W_in = Win;
  a.Wn = Wn;
  a.W_out = Wout;
  a.ctl = b->ctl;
  a.stats = b->stats;
  return a;
}

// Enqueue one SSPRK3 step of every problem on stream s with tile variant v.
int enqueue_batch_step(wcns_batch *b, double *W, double cfl, double *t_acc, int v, int grid, cudaStream_t s) {
  batch_begin_kernel<<<(b->nprob + 255) / 256, 256, 0, s>>>(b->nprob, b->inv_dx, b->dt, b->smax, cfl, t_acc);
  b->launches++;
  if (cudaGetLastError() != cudaSuccess) return WCNS_E_CUDA;
  for (int st = 0; st < 3; ++st) {
    const double *Win = st == 0 ? W : (st == 1 ? b->W1 : b->W2);
    double *Wout = st == 0 ? b->W1 : (st == 1 ? b->W2 : W);
    SweepArgs a = stage_args(b, st, Win, Wout, W);
    // only the last stage's wave-speed maxima feed the next step's dt
    BatchArgs ba = batch_args(b, v, st == 2 ? b->smax : b->smax_scratch);
    const Variant &var = kVariants[v];
    const BatchLauncher launch = b->opt.precision == WCNS_MIXED ? var.mixed : var.fp64;
    if (!launch) return WCNS_E_UNSUPPORTED;
    cudaError_t e = launch(a, ba, grid, s);
    b->launches++;
    if (e != cudaSuccess) return WCNS_E_CUDA;
  }
  return WCNS_OK;
}

int launch_batch_reduce(wcns_batch *b, const double *W, cudaStream_t s) {
  if (cudaMemsetAsync(b->smax, 0, sizeof(unsigned long long) * b->nprob, s) != cudaSuccess) return WCNS_E_CUDA;
  BatchArgs ba = batch_args(b, 1, b->smax);
  const int grid = b->sms * 8 < ba.ntiles ? b->sms * 8 : ba.ntiles;
  batch_reduce_kernel<<<grid > 0 ? grid : 1, 128, 0, s>>>(W, b->total, b->eos, ba, kVariants[1].tm - 1);
  b->launches++;
  return cudaGetLastError() == cudaSuccess ? WCNS_OK : WCNS_E_CUDA;
}

void drop_graph(wcns_batch *b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = NULL;
  b->graph_W = NULL;
}

// ---------------------------------------------------------------------------
// 2D batches: host side.
// ---------------------------------------------------------------------------
Batch2Args batch2_args(wcns_batch *b, int dir) {
  Batch2Args a;
  a.offsets = b->offsets;
  a.nx = b->nx2;
  a.ny = b->ny2;
  a.inv_dx = b->inv_dx2;
  a.dt = b->dt;
  a.smax = b->smax2;
  a.l_unit = b->l_unit2;
  a.tile_prob = b->tl_prob[dir];
  a.tile_first = b->tl_first[dir];
  a.tile_line = b->tl_line[dir];
  a.ntiles = b->ntl[dir];
  return a;
}

// The sweep of direction d, k-th in the stage's order, of SSPRK3 stage s:
// the single-grid orchestration (wcns_api.cu) with per-problem scalars
// taken from the tables by the geometry policy.
SweepArgs batch2_stage_args(wcns_batch *b, int s, int k, int d, const double *Win, double *Wout, const double *Wn) {
  SweepArgs a;
  memset(&a, 0, sizeof(a));
  a.n[0] = a.n[1] = a.n[2] = 1;
  a.ncell = b->total;
  a.bc_lo = b->bc[d][0];
  a.bc_hi = b->bc[d][1];
  a.eos = b->eos;
  a.tol.eps_ar = b->opt.eps_ar;
  a.tol.eps_a = b->opt.eps_a;
  a.tol.eps_rc = b->opt.eps_rc;
  a.tol.hs_ar = b->opt.hs_ar;
  a.tol.hs_a = b->opt.hs_a;
  a.tol.hs_rc = b->opt.hs_rc;
  set_cert(a.tol);
  a.eps_is = b->opt.eps_is;
  a.eps_is32 = (float)fmax(b->opt.eps_is, 1e-30);
  a.scheme = b->opt.scheme;
  a.stage = s;
  a.W_in = Win;
  a.Wn = Wn;
  a.L = b->L2;
  a.ctl = b->ctl;
  a.stats = b->stats;
  const bool mixed = b->opt.precision == WCNS_MIXED;
  if (mixed) {
    a.node_p = b->node_p;
    a.node_ir = b->node_ir;
    a.node_c = b->node_c;
    a.node_ok = b->node_ok;
    a.node_write = k == 0;
    a.node_read = k != 0;
  }
  if (k == 0) {
    a.epilogue = EPI_WRITE;
    a.l_raw = mixed;  // mixed: the raw difference, the combine applies 1/dx_d0
  } else {
    const double ra[3] = {0.0, 0.75, 1.0 / 3.0};
    const double rb[3] = {1.0, 0.25, 2.0 / 3.0};
    a.epilogue = EPI_COMBINE;
    a.read_L = 1;
    a.rk_a = ra[s];
    a.rk_b = rb[s];
    a.W_out = Wout;
  }
  return a;
}

// The sweep order of one stage: x then y in FP64; in the mixed path the
// order of mixed_first_dir, as for a single grid.
int batch2_dir(const wcns_batch *b, int k) {
  return (b->opt.precision == WCNS_MIXED && mixed_first_dir(2) != 0) ? 1 - k : k;
}

cudaError_t batch2_launch(wcns_batch *b, int d, const SweepArgs &a, const Batch2Args &ba, int grid, cudaStream_t s) {
  const bool mixed = b->opt.precision == WCNS_MIXED;
  if (d == 0) return mixed ? launch_batch2<true, 0>(a, ba, grid, s) : launch_batch2<false, 0>(a, ba, grid, s);
  return mixed ? launch_batch2<true, 1>(a, ba, grid, s) : launch_batch2<false, 1>(a, ba, grid, s);
}

int enqueue_batch2_step(wcns_batch *b, double *W, double cfl, double *t_acc, int bps, cudaStream_t s) {
  batch2_begin_kernel<<<(b->nprob + 255) / 256, 256, 0, s>>>(b->nprob, b->inv_dx2, b->dt, b->smax2, cfl, t_acc);
  b->launches++;
  if (cudaGetLastError() != cudaSuccess) return WCNS_E_CUDA;
  for (int st = 0; st < 3; ++st) {
    const double *Win = st == 0 ? W : (st == 1 ? b->W1 : b->W2);
    double *Wout = st == 0 ? b->W1 : (st == 1 ? b->W2 : W);
    for (int k = 0; k < 2; ++k) {
      const int d = batch2_dir(b, k);
      const SweepArgs a = batch2_stage_args(b, st, k, d, Win, Wout, W);
      const Batch2Args ba = batch2_args(b, d);
      int grid = b->sms * bps;
      if (grid > ba.ntiles) grid = ba.ntiles;
      if (grid < 1) grid = 1;
      const cudaError_t e = batch2_launch(b, d, a, ba, grid, s);
      b->launches++;
      if (e != cudaSuccess) return WCNS_E_CUDA;
    }
  }
  return WCNS_OK;
}

int launch_batch2_reduce(wcns_batch *b, const double *W, cudaStream_t s) {
  if (cudaMemsetAsync(b->smax2, 0, sizeof(unsigned long long) * 8 * (size_t)b->nprob, s) != cudaSuccess)
    return WCNS_E_CUDA;
  const Batch2Args ba = batch2_args(b, 0);
  int grid = b->sms * 8 < ba.ntiles ? b->sms * 8 : ba.ntiles;
  if (grid < 1) grid = 1;
  batch2_reduce_kernel<<<grid, 256, 0, s>>>(W, b->total, b->eos, ba);
  b->launches++;
  return cudaGetLastError() == cudaSuccess ? WCNS_OK : WCNS_E_CUDA;
}

// 2D autotuner: time two steps for each persistent grid of 1 .. the
// occupancy limit blocks per SM on a copy of the state; keep the fastest.
int autotune2(wcns_batch *b, const double *W, double cfl) {
  const size_t bytes = sizeof(double) * 6 * (size_t)b->total;
  DevStats saved;
  cudaStreamSynchronize(b->stream);
  cudaMemcpy(&saved, b->stats, sizeof(saved), cudaMemcpyDeviceToHost);
  const bool mixed = b->opt.precision == WCNS_MIXED;
  int occ = mixed ? batch2_max_blocks_per_sm<true, 0>() : batch2_max_blocks_per_sm<false, 0>();
  const int occ1 = mixed ? batch2_max_blocks_per_sm<true, 1>() : batch2_max_blocks_per_sm<false, 1>();
  if (occ1 < occ) occ = occ1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bb = 1;
  for (int bps = 1; bps <= occ && bps <= 8; ++bps) {
    cudaMemcpyAsync(b->Wtrial, W, bytes, cudaMemcpyDeviceToDevice, b->cap);
    if (launch_batch2_reduce(b, b->Wtrial, b->cap)) continue;
    if (enqueue_batch2_step(b, b->Wtrial, cfl, NULL, bps, b->cap)) continue;  // warm
    cudaEventRecord(e0, b->cap);
    for (int r = 0; r < 2; ++r) enqueue_batch2_step(b, b->Wtrial, cfl, NULL, bps, b->cap);
    cudaEventRecord(e1, b->cap);
    if (cudaEventSynchronize(e1) != cudaSuccess) continue;
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) {
      best = ms;
      bb = bps;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(b->cap);
  cudaMemcpy(b->stats, &saved, sizeof(saved), cudaMemcpyHostToDevice);
  if (cudaGetLastError() != cudaSuccess) return WCNS_E_CUDA;
  b->grid = bb;  // 2D: blocks per SM of the persistent sweeps
  b->tuned = 1;
  return WCNS_OK;
}

// Autotuner: time one step of every (tile length, blocks per SM) candidate
// on a copy of the state and keep the fastest.
int autotune(wcns_batch *b, const double *W, double cfl) {
  const size_t bytes = sizeof(double) * 5 * (size_t)b->total;
  double *trial = b->Wtrial;  // allocated at create: tuning allocates nothing
  DevStats saved;
  cudaStreamSynchronize(b->stream);
  cudaMemcpy(&saved, b->stats, sizeof(saved), cudaMemcpyDeviceToHost);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bv = b->opt.precision == WCNS_MIXED ? 4 : 1, bg = b->sms;  // fallbacks: 127-cell tiles
  for (int v = 0; v < kNumVariants; ++v) {
    const bool mixed = b->opt.precision == WCNS_MIXED;
    if (!(mixed ? kVariants[v].mixed : kVariants[v].fp64)) continue;
    const int occ = mixed ? kVariants[v].occm() : kVariants[v].occ64();
    for (int bps = 1; bps <= occ && bps <= 16; bps = (bps * 2 > occ && bps < occ) ? occ : bps * 2) {
      int grid = b->sms * bps;
      if (grid > b->ntiles[v]) grid = b->ntiles[v];
      cudaMemcpyAsync(trial, W, bytes, cudaMemcpyDeviceToDevice, b->cap);
      if (launch_batch_reduce(b, trial, b->cap)) continue;
      if (enqueue_batch_step(b, trial, cfl, NULL, v, grid, b->cap)) continue;  // warm
      cudaEventRecord(e0, b->cap);
      for (int r = 0; r < 2; ++r) enqueue_batch_step(b, trial, cfl, NULL, v, grid, b->cap);
      cudaEventRecord(e1, b->cap);
      if (cudaEventSynchronize(e1) != cudaSuccess) continue;
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        bv = v;
        bg = grid;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(b->cap);
  cudaMemcpy(b->stats, &saved, sizeof(saved), cudaMemcpyHostToDevice);
  if (cudaGetLastError() != cudaSuccess) return WCNS_E_CUDA;
  b->variant = bv;
  b->grid = bg;
  b->tuned = 1;
  return WCNS_OK;
}

}  // namespace

extern "C" {

int wcns_batch_create(int nprob, const int *ncells, const double *lo, const double *hi, int bc_lo, int bc_hi,
                      double gamma_g, double gamma_l, double pinf_l, wcns_batch **out) {
  if (!out) return WCNS_E_INVALID_ARG;
  *out = NULL;
  if (nprob < 1 || !ncells || !lo || !hi) return WCNS_E_INVALID_ARG;
  if (!(gamma_g > 1.0) || !(gamma_l > 1.0) || !(pinf_l >= 0.0) || !(gamma_g <= gamma_l)) return WCNS_E_INVALID_ARG;
  if ((bc_lo != WCNS_BC_TRANSMISSIVE && bc_lo != WCNS_BC_PERIODIC && bc_lo != WCNS_BC_SYMMETRY) ||
      (bc_hi != WCNS_BC_TRANSMISSIVE && bc_hi != WCNS_BC_PERIODIC && bc_hi != WCNS_BC_SYMMETRY) ||
      ((bc_lo == WCNS_BC_PERIODIC) != (bc_hi == WCNS_BC_PERIODIC)))
    return WCNS_E_INVALID_ARG;
  const bool sym = bc_lo == WCNS_BC_SYMMETRY || bc_hi == WCNS_BC_SYMMETRY;
  std::vector<long long> offs(nprob);
  std::vector<double> idx(nprob);
  long long total = 0;
  for (int k = 0; k < nprob; ++k) {
    if (ncells[k] < 1 || !(hi[k] > lo[k]) || !isfinite(hi[k] - lo[k]) || (sym && ncells[k] < 3))
      return WCNS_E_INVALID_ARG;
    offs[k] = total;
    total += ncells[k];
    idx[k] = 1.0 / ((hi[k] - lo[k]) / ncells[k]);  // same rounding as the single-grid handle
  }
  wcns_batch *b = (wcns_batch *)calloc(1, sizeof(wcns_batch));
  if (!b) return WCNS_E_CUDA;
  b->ndim = 1;
  b->nprob = nprob;
  b->total = total;
  b->bc_lo = bc_lo;
  b->bc_hi = bc_hi;
  b->eos = make_eos(gamma_g, gamma_l, pinf_l);
  wcns_default_options(&b->opt);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  if (b->sms < 1) b->sms = 1;
  cudaError_t e = cudaSuccess;
  const size_t sbytes = sizeof(double) * 5 * (size_t)total;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&b->offsets, sizeof(long long) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->ncell, sizeof(int) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->inv_dx, sizeof(double) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->dt, sizeof(double) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->smax, sizeof(unsigned long long) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->smax_scratch, sizeof(unsigned long long) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->W1, sbytes);
  if (e == cudaSuccess) e = cudaMalloc(&b->W2, sbytes);
  if (e == cudaSuccess) e = cudaMalloc(&b->Wtrial, sbytes);
  if (e == cudaSuccess) e = cudaMalloc(&b->stats, sizeof(DevStats));
  if (e == cudaSuccess) e = cudaMalloc(&b->ctl, sizeof(StepCtl));
  if (e == cudaSuccess) e = cudaMemset(b->stats, 0, sizeof(DevStats));
  if (e == cudaSuccess) e = cudaMemset(b->ctl, 0, sizeof(StepCtl));
  if (e == cudaSuccess) e = cudaMemcpy(b->offsets, offs.data(), sizeof(long long) * nprob, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->ncell, ncells, sizeof(int) * nprob, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->inv_dx, idx.data(), sizeof(double) * nprob, cudaMemcpyHostToDevice);
  // work lists, one per tile length (tiles of TM midpoints cover TM-1 cells)
  for (int v = 0; v < kNumVariants && e == cudaSuccess; ++v) {
    std::vector<int> tp, tf;
    const int per = kVariants[v].tm - 1;
    for (int k = 0; k < nprob; ++k)
      for (int c = 0; c < ncells[k]; c += per) {
        tp.push_back(k);
        tf.push_back(c);
      }
    b->ntiles[v] = (int)tp.size();
    e = cudaMalloc(&b->tile_prob[v], sizeof(int) * tp.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->tile_first[v], sizeof(int) * tf.size());
    if (e == cudaSuccess) e = cudaMemcpy(b->tile_prob[v], tp.data(), sizeof(int) * tp.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->tile_first[v], tf.data(), sizeof(int) * tf.size(), cudaMemcpyHostToDevice);
  }
  b->variant = 1;
  b->grid = b->sms;
  if (e != cudaSuccess) {
    wcns_batch_destroy(b);
    return WCNS_E_CUDA;
  }
  *out = b;
  return WCNS_OK;
}

int wcns_batch_create_grids(int ndim, int nprob, const int *n, const double *lo, const double *hi,
                            const wcns_bcs *bcs, double gamma_g, double gamma_l, double pinf_l, wcns_batch **out) {
  if (!out) return WCNS_E_INVALID_ARG;
  *out = NULL;
  if (nprob < 1 || !n || !lo || !hi || !bcs) return WCNS_E_INVALID_ARG;
  if (ndim == 1)
    return wcns_batch_create(nprob, n, lo, hi, bcs->kind[0][0], bcs->kind[0][1], gamma_g, gamma_l, pinf_l, out);
  if (ndim != 2) return WCNS_E_UNSUPPORTED;
  if (!(gamma_g > 1.0) || !(gamma_l > 1.0) || !(pinf_l >= 0.0) || !(gamma_g <= gamma_l) || !isfinite(gamma_g) ||
      !isfinite(gamma_l) || !isfinite(pinf_l))
    return WCNS_E_INVALID_ARG;
  bool sym[2];
  for (int d = 0; d < 2; ++d) {
    for (int sd = 0; sd < 2; ++sd) {
      const int k = bcs->kind[d][sd];
      if (k != WCNS_BC_TRANSMISSIVE && k != WCNS_BC_PERIODIC && k != WCNS_BC_SYMMETRY) return WCNS_E_INVALID_ARG;
    }
    if ((bcs->kind[d][0] == WCNS_BC_PERIODIC) != (bcs->kind[d][1] == WCNS_BC_PERIODIC)) return WCNS_E_INVALID_ARG;
    sym[d] = bcs->kind[d][0] == WCNS_BC_SYMMETRY || bcs->kind[d][1] == WCNS_BC_SYMMETRY;
  }
  std::vector<long long> offs(nprob);
  std::vector<double> idx(2 * (size_t)nprob), lunit(nprob);
  long long total = 0;
  for (int k = 0; k < nprob; ++k) {
    for (int d = 0; d < 2; ++d) {
      const int nk = n[2 * k + d];
      const double L = hi[2 * k + d] - lo[2 * k + d];
      if (nk < 1 || nk > (1 << 20) || !(L > 0.0) || !isfinite(L) || (sym[d] && nk < 3)) return WCNS_E_INVALID_ARG;
      idx[2 * k + d] = 1.0 / (L / nk);  // the single grid's rounding of 1/dx
    }
    offs[k] = total;
    total += (long long)n[2 * k] * n[2 * k + 1];
    if (total > (1ll << 34)) return WCNS_E_INVALID_ARG;
    lunit[k] = idx[2 * k + mixed_first_dir(2)];
  }
  wcns_batch *b = (wcns_batch *)calloc(1, sizeof(wcns_batch));
  if (!b) return WCNS_E_CUDA;
  b->ndim = 2;
  b->nprob = nprob;
  b->total = total;
  for (int d = 0; d < 2; ++d)
    for (int sd = 0; sd < 2; ++sd) b->bc[d][sd] = bcs->kind[d][sd];
  b->eos = make_eos(gamma_g, gamma_l, pinf_l);
  wcns_default_options(&b->opt);
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  if (b->sms < 1) b->sms = 1;
  std::vector<int> nx(nprob), ny(nprob);
  for (int k = 0; k < nprob; ++k) {
    nx[k] = n[2 * k];
    ny[k] = n[2 * k + 1];
  }
  cudaError_t e = cudaSuccess;
  const size_t sbytes = sizeof(double) * 6 * (size_t)total;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&b->offsets, sizeof(long long) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->nx2, sizeof(int) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->ny2, sizeof(int) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->inv_dx2, sizeof(double) * 2 * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->l_unit2, sizeof(double) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->dt, sizeof(double) * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->smax2, sizeof(unsigned long long) * 8 * nprob);
  if (e == cudaSuccess) e = cudaMalloc(&b->W1, sbytes);
  if (e == cudaSuccess) e = cudaMalloc(&b->W2, sbytes);
  if (e == cudaSuccess) e = cudaMalloc(&b->L2, sbytes);
  if (e == cudaSuccess) e = cudaMalloc(&b->Wtrial, sbytes);
  if (e == cudaSuccess) {
    // node cache of the mixed sweeps: [p | 1/rho] doubles, [c | bits] 32-bit words
    e = cudaMalloc(&b->node_p, (2 * sizeof(double) + 2 * sizeof(float)) * (size_t)total);
    if (e == cudaSuccess) {
      b->node_ir = b->node_p + total;
      b->node_c = (float *)(b->node_ir + total);
      b->node_ok = (unsigned int *)(b->node_c + total);
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&b->stats, sizeof(DevStats));
  if (e == cudaSuccess) e = cudaMalloc(&b->ctl, sizeof(StepCtl));
  if (e == cudaSuccess) e = cudaMemset(b->stats, 0, sizeof(DevStats));
  if (e == cudaSuccess) e = cudaMemset(b->ctl, 0, sizeof(StepCtl));
  if (e == cudaSuccess) e = cudaMemset(b->smax2, 0, sizeof(unsigned long long) * 8 * nprob);
  if (e == cudaSuccess) e = cudaMemcpy(b->offsets, offs.data(), sizeof(long long) * nprob, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->nx2, nx.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->ny2, ny.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->inv_dx2, idx.data(), sizeof(double) * 2 * nprob, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->l_unit2, lunit.data(), sizeof(double) * nprob, cudaMemcpyHostToDevice);
  // work lists: x tiles of TL rows x (TM - 1) cells, y tiles of TL columns x (TM - 1) cells
  for (int d = 0; d < 2 && e == cudaSuccess; ++d) {
    const int TL = d == 0 ? Batch2TileX::TL : Batch2TileY::TL;
    const int per = (d == 0 ? Batch2TileX::TM : Batch2TileY::TM) - 1;
    std::vector<int> tp, tf, tl;
    for (int k = 0; k < nprob; ++k) {
      const int nlines = d == 0 ? ny[k] : nx[k], nalong = d == 0 ? nx[k] : ny[k];
      for (int l0 = 0; l0 < nlines; l0 += TL)
        for (int c = 0; c < nalong; c += per) {
          tp.push_back(k);
          tf.push_back(c);
          tl.push_back(l0);
        }
    }
    if (tp.size() > (size_t)0x7FFFFFFF) e = cudaErrorInvalidValue;
    b->ntl[d] = (int)tp.size();
    if (e == cudaSuccess) e = cudaMalloc(&b->tl_prob[d], sizeof(int) * tp.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->tl_first[d], sizeof(int) * tp.size());
    if (e == cudaSuccess) e = cudaMalloc(&b->tl_line[d], sizeof(int) * tp.size());
    if (e == cudaSuccess) e = cudaMemcpy(b->tl_prob[d], tp.data(), sizeof(int) * tp.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->tl_first[d], tf.data(), sizeof(int) * tf.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->tl_line[d], tl.data(), sizeof(int) * tl.size(), cudaMemcpyHostToDevice);
  }
  b->grid = 1;
  if (e != cudaSuccess) {
    wcns_batch_destroy(b);
    return WCNS_E_CUDA;
  }
  *out = b;
  return WCNS_OK;
}

int wcns_batch_set_options(wcns_batch *b, const wcns_options *o) {
  if (!b || !o) return WCNS_E_INVALID_ARG;
  if (o->precision != WCNS_FP64 && o->precision != WCNS_MIXED) return WCNS_E_INVALID_ARG;
  if (o->scheme < 0 || o->scheme > 2 || !valid_tolerances(*o)) return WCNS_E_INVALID_ARG;
  if (b->opt.precision != o->precision || b->opt.scheme != o->scheme) b->tuned = 0;
  b->opt = *o;
  b->stream = (cudaStream_t)o->stream;
  drop_graph(b);
  return WCNS_OK;
}

int wcns_batch_advance(wcns_batch *b, double *W, int nsteps, double cfl, double *t_out) {
  if (!b || !W || nsteps < 0 || !(cfl > 0.0 && cfl <= 1.0)) return WCNS_E_INVALID_ARG;
  if (nsteps == 0) return WCNS_OK;
  if (!b->tuned) {
    int st = b->ndim == 2 ? autotune2(b, W, cfl) : autotune(b, W, cfl);
    if (st) return st;
    drop_graph(b);
  }
  // order after the caller's pending work
  if (cudaEventRecord(b->ev_in, b->stream) != cudaSuccess) return WCNS_E_CUDA;
  if (cudaStreamWaitEvent(b->cap, b->ev_in, 0) != cudaSuccess) return WCNS_E_CUDA;
  batch_snapshot_kernel<<<1, 1, 0, b->cap>>>(b->stats, b->ctl);
  b->launches++;
  if (cudaGetLastError() != cudaSuccess) return WCNS_E_CUDA;
  int st = b->ndim == 2 ? launch_batch2_reduce(b, W, b->cap) : launch_batch_reduce(b, W, b->cap);
  if (st) return st;
  if (!b->graph || b->graph_W != W || b->graph_cfl != cfl || b->graph_t != t_out) {
    drop_graph(b);
    cudaGraph_t g;
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return WCNS_E_CUDA;
    const long long before = b->launches;
    st = b->ndim == 2 ? enqueue_batch2_step(b, W, cfl, t_out, b->grid, b->cap)
                      : enqueue_batch_step(b, W, cfl, t_out, b->variant, b->grid, b->cap);
    b->launches = before;  // counted when replayed
    cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (e == cudaSuccess && st) cudaGraphDestroy(g);  // a partial capture is never launched
    if (st || e != cudaSuccess) return st ? st : WCNS_E_CUDA;
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      b->graph = NULL;
      return WCNS_E_CUDA;
    }
    b->graph_W = W;
    b->graph_cfl = cfl;
    b->graph_t = t_out;
  }
  for (int k = 0; k < nsteps; ++k) {
    if (cudaGraphLaunch(b->graph, b->cap) != cudaSuccess) return WCNS_E_CUDA;
    b->launches += 1 + 3 * b->ndim;
  }
  if (cudaEventRecord(b->ev_out, b->cap) != cudaSuccess) return WCNS_E_CUDA;
  if (cudaStreamWaitEvent(b->stream, b->ev_out, 0) != cudaSuccess) return WCNS_E_CUDA;
  // status: the counters against their snapshot (synchronises)
  StepCtl c;
  DevStats s;
  if (cudaMemcpyAsync(&c, b->ctl, sizeof(c), cudaMemcpyDeviceToHost, b->cap) != cudaSuccess) return WCNS_E_CUDA;
  if (cudaMemcpyAsync(&s, b->stats, sizeof(s), cudaMemcpyDeviceToHost, b->cap) != cudaSuccess) return WCNS_E_CUDA;
  if (cudaStreamSynchronize(b->cap) != cudaSuccess) return WCNS_E_CUDA;
  return status_from_counts(c, s, WCNS_OK, WCNS_E_NONFINITE, WCNS_E_INADMISSIBLE);
}

int wcns_batch_get_stats(wcns_batch *b, wcns_stats *out) {
  if (!b || !out) return WCNS_E_INVALID_ARG;
  DevStats s;
  if (cudaStreamSynchronize(b->cap) != cudaSuccess) return WCNS_E_CUDA;
  if (cudaMemcpy(&s, b->stats, sizeof(s), cudaMemcpyDeviceToHost) != cudaSuccess) return WCNS_E_CUDA;
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

long long wcns_batch_total_cells(const wcns_batch *b) { return b ? b->total : 0; }
long long wcns_batch_launch_count(const wcns_batch *b) { return b ? b->launches : 0; }

int wcns_batch_tuning(const wcns_batch *b, int *tile_cells, int *grid) {
  if (!b) return WCNS_E_INVALID_ARG;
  if (b->ndim == 2) {  // x tiles' cells; persistent blocks of the sweeps (capped by their work lists)
    if (tile_cells) *tile_cells = Batch2TileX::TL * (Batch2TileX::TM - 1);
    if (grid) *grid = b->sms * b->grid;
    return b->tuned ? WCNS_OK : WCNS_E_UNSUPPORTED;
  }
  if (tile_cells) *tile_cells = kVariants[b->variant].tm - 1;
  if (grid) *grid = b->grid;
  return b->tuned ? WCNS_OK : WCNS_E_UNSUPPORTED;
}

void wcns_batch_destroy(wcns_batch *b) {
  if (!b) return;
  if (b->cap) cudaStreamSynchronize(b->cap);
  drop_graph(b);
  for (int v = 0; v < kNumVariants; ++v) {
    cudaFree(b->tile_prob[v]);
    cudaFree(b->tile_first[v]);
  }
  for (int d = 0; d < 2; ++d) {
    cudaFree(b->tl_prob[d]);
    cudaFree(b->tl_first[d]);
    cudaFree(b->tl_line[d]);
  }
  cudaFree(b->nx2);
  cudaFree(b->ny2);
  cudaFree(b->inv_dx2);
  cudaFree(b->l_unit2);
  cudaFree(b->smax2);
  cudaFree(b->L2);
  cudaFree(b->node_p);
  cudaFree(b->offsets);
  cudaFree(b->ncell);
  cudaFree(b->inv_dx);
  cudaFree(b->dt);
  cudaFree(b->smax);
  cudaFree(b->smax_scratch);
  cudaFree(b->W1);
  cudaFree(b->W2);
  cudaFree(b->Wtrial);
  cudaFree(b->stats);
  cudaFree(b->ctl);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->cap) cudaStreamDestroy(b->cap);
  free(b);
}

}  // extern "C"
