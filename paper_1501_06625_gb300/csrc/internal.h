// internal.h -- host-side structures of libph shared by its translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <utility>
#include <string>
#include <vector>

#include "ph.h"

// Device allocations of the library, counted against the cap set by
// ph_set_memory_limit (api.cu): beyond it an allocation fails with
// cudaErrorMemoryAllocation, as on a full device.
cudaError_t ph_dev_alloc(void **p, size_t bytes);
void ph_dev_free(void *p, size_t bytes);

// A growable device buffer owned by a context or a system.
struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) ph_dev_free(p, cap ? cap : 16);
    p = nullptr;
    cap = 0;
    cudaError_t e = ph_dev_alloc(&p, bytes ? bytes : 16);
    if (e == cudaSuccess) cap = bytes;
    return e;
  }
  void release() {
    if (p) ph_dev_free(p, cap ? cap : 16);
    p = nullptr;
    cap = 0;
  }
  template <class T> T *as() const { return (T *)p; }
};

// Device-side state of one tracked path and of its current corrector run.
// Lives in device memory; the step kernels read and update it.
struct PathState {
  // step-size controller (Fig. 3)
  ph_ctrl_state ctrl;
  // the step being tried
  double t_new;
  int32_t hist_count, hist_head;
  // corrector (Fig. 2)
  int32_t nt_done, nt_success, nt_iters, nt_updates;
  double last_res, res, dxn;
  unsigned long long res_bits, dx_bits, x_bits;
  // path statistics
  int32_t steps, accepted, rejected, newton_iters, updates, log_len;
  double res_last, dx_last;
  // set when a bounded device wait ran out
  int32_t timeout, mgs_status;
  // grid barrier of the cooperative kernels
  unsigned int bar_count, bar_gen;
  // the MGS solve: epoch of its pivot flags, blocks finished
  int32_t mgs_epoch;
  unsigned int mgs_done;
  int32_t iterations;           // passes of the graph's step body
  // kernel gates: a kernel does nothing while its flag is set
  int32_t skip_step, skip_nt;
  double t_dev[4];              // t of the step, L limbs
  double hist_t[16];            // t of the accepted points in the history ring
  // the precision form (lin_prec 1): the precision of the current solve (0
  // working, 1 double), the scale exponent of the right-hand side, the
  // escalation state of the step, and the gates of the two kernel sets
  int32_t lin, scale_e, force, escalate, onpath, retry, pass, linear, wp_rest;
  double dxn2;                  // the update before the last one (this pass)
  int32_t gate_wp, gate_lp;
  int32_t solves_f64, escalated;
  double cond;
};

// Measured times (ms) of the MGS variants of one shape: grid, cluster, tiled
// (the best row-block count, tile_R); 1e30 where a variant does not apply.
struct MgsTimes {
  float ms[3] = {1e30f, 1e30f, 1e30f};
  int tile_R = 0;
};

struct ph_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  std::string err;
  DevBuf in_x, in_gamma, in_t, in_J, in_rhs;       // staged host inputs
  DevBuf out_h, out_J, out_dx;                      // staged outputs
  DevBuf slots, ptab, scal, A, R, nrm2, irkk, dxv, state, hist, xw, logbuf, ystage, flags, spow;
  DevBuf bws, bq, bx0, bxo, bstats, blog, btune;    // many-path tracking
  // the MGS variant chosen for each shape (key (L, N, n)): 0 the grid kernel,
  // C > 0 the cluster kernel with C CTAs; scratch buffers of the choice
  std::map<long long, int> mgs_variant;
  std::map<long long, MgsTimes> mgs_times;
  DevBuf tuneA, tuneW, tuneN, tuneF, tuneX, tuneS, mgs_part;
  // limit of every bounded device-side wait (ns), and the pivot whose
  // hand-off the solves withhold (test support; -1: none)
  unsigned long long wait_ns = 2000000000ull;
  int withhold = -1;
};

// A loaded polynomial system: the instruction layout of Section 3.2 (terms
// sorted by their number of variables, position-major arrays so consecutive
// threads read consecutive addresses) plus the summation lists.
struct ph_system {
  ph_ctx *ctx = nullptr;
  // unique per load in this process: caches key on it, never on the address,
  // which a later load may reuse after ph_system_free
  uint64_t serial = 0;
  int L = 2, N = 0, n = 0, M = 0, Mp = 0, maxv = 0, emax = 1;
  int nout = 0;                 // n*N Jacobian entries + N values
  int max_contrib = 0;          // longest summation list
  DevBuf poly, nv, vidx, vexp, coeff, deg, out_ptr, out_slot;
  // one byte per polynomial: 1 if it has no terms (the rows a start system
  // leaves to f when the tracker holds them fixed, ph_track_params.fixed_rows)
  DevBuf zero_rows;
  // sorted terms [s0, s1) differentiated with `lanes` threads per monomial
  struct Bucket { int s0, s1, lanes; };
  std::vector<Bucket> buckets;
  std::vector<int> h_deg;
  int max_deg = 0;
  // lanes per output of the summation kernel (#Th of the paper's Section 3.3),
  // chosen by timing on the first evaluation (0: not yet), and the times (ms)
  // of 1, 2, 4, 8, 16 and 32 lanes
  mutable int sum_lanes = 0;
  mutable float sum_ms[6] = {-1, -1, -1, -1, -1, -1};
  // the same choice for the summation inside the many-path and serving
  // kernels (one block per path), timed on a batch of that kernel: 0 until
  // timed (4 lanes are used), with the times (ms per launch) of 1 .. 32 lanes
  mutable int block_lanes = 0;
  mutable float block_ms[6] = {-1, -1, -1, -1, -1, -1};
};

// ---- helpers (api.cu)
ph_status ph_fail(ph_ctx *ctx, ph_status st, const std::string &msg);
ph_status ph_cuda_fail(ph_ctx *ctx, cudaError_t e, const char *where);
bool ph_is_device_ptr(const void *p);

#define PH_CUDA(ctx, call)                                       \
  do {                                                           \
    cudaError_t e__ = (call);                                    \
    if (e__ != cudaSuccess) return ph_cuda_fail(ctx, e__, #call); \
  } while (0)

// ---- kernels' host launchers
// eval.cu: values and Jacobian of the homotopy into device buffers.
//   J: plane stride Jplane (doubles between limb/part planes), leading dim ldJ
//   h: [2L][N] (may be null); rhs: -h into a plane-strided column (may be null)
//   t: L limbs on the device; gamma: [2L] on the device or null (f alone)
//   skip: device flag; the kernels do nothing while *skip != 0 (may be null)
//   res_bits: max |h_i| (leading limbs, double bits) accumulated (may be null)
//   fixed: one byte per row, rows held fixed (h_i = f_i), or null
cudaError_t ph_eval_launch(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                           const double *gamma, int k, const double *t, const double *x,
                           double *h, double *J, long ldJ, long Jplane,
                           double *rhs, long rhs_plane, const int *skip,
                           unsigned long long *res_bits, const uint8_t *fixed = nullptr);

// the same, launching only the kernels selected by `parts`
// (1 = power table and factors, 2 = monomial AD, 4 = summation)
cudaError_t ph_eval_launch_part(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                                const double *gamma, int k, const double *t, const double *x,
                                double *h, double *J, long ldJ, long Jplane, double *rhs,
                                long rhs_plane, const int *skip, unsigned long long *res_bits,
                                int parts, const uint8_t *fixed = nullptr);

// eval.cu: h alone in the working precision (no derivatives): -h's leading
// limbs to rhs ([re|im], planes rhs_plane apart), max |h_i| to *res_bits.
cudaError_t ph_eval_values_launch(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                                  const double *gamma, int k, const double *t, const double *x,
                                  double *rhs, long rhs_plane, const int *skip,
                                  unsigned long long *res_bits, const uint8_t *fixed = nullptr);

// eval.cu: the Jacobian alone in IEEE double from the leading limbs of every
// input (x, t, gamma, the coefficients), in the one-limb layout.
cudaError_t ph_eval_launch_f64(ph_ctx *ctx, const ph_system *f, const ph_system *g,
                               const double *gamma, int k, const double *t, const double *x,
                               double *J, long ldJ, long Jplane, const int *skip,
                               const uint8_t *fixed = nullptr);

// eval.cu: the summation kernel's lanes per output for f (and g), measured
// on the first evaluation outside a stream capture (called before a capture).
void ph_sum_tune(ph_ctx *ctx, const ph_system *f, const ph_system *g);

// mgs.cu: least squares on the augmented matrix A = [J | rhs] held in
//   A (plane stride (n+1)*ldA, leading dim ldA); dx [2L][n] out;
//   st->dx_bits: max |dx_i| accumulated; resid: ||residual||_2 (may be null);
//   ctx->nrm2[k] (k < n) ends as the leading limb of r_kk^2 with either variant.
//   The pivot flags (ctx->flags, n+1 ints) must be zero when the state's
//   mgs_epoch is zero: zero both at the start of every call.
cudaError_t ph_mgs_launch(ph_ctx *ctx, int L, int N, int n, double *A, long ldA, double *dx,
                          PathState *st, const int *skip, double *resid);

int ph_mgs_grid(ph_ctx *ctx, int L, int N, int n);

// The MGS variant for a shape, measured once per context on a scratch matrix
// (outside stream capture; during a capture an unmeasured shape gets the grid
// kernel): 0 = grid kernel, C > 0 = cluster kernel with C CTAs.
int ph_mgs_tune(ph_ctx *ctx, int L, int N, int n);

// mgs_cluster.cu: the same solve on one thread-block cluster (A is read, not
// modified).  ph_mgs_cluster_size: 16 or 8 CTAs, or 0 if the matrix does not
// fit in a cluster's shared memory.
int ph_mgs_cluster_size(int L, int N, int n);

// mgs_tile.cu: the same solve as a tiled right-looking MGS (R row blocks x
// column groups, one grid barrier per pivot).  ph_mgs_tile_grid: its blocks
// for R row blocks, 0 if R does not fit; ph_mgs_tile_part: doubles of its
// partial-sum buffer.
int ph_mgs_tile_grid(int sm_count, int L, int N, int n, int R);
long ph_mgs_tile_part(int L, int n, int R);
cudaError_t ph_mgs_tile_launch(int sm_count, cudaStream_t stream, int L, int N, int n, int R,
                               double *A, long ldA, double *W, double *nrm2, double *part,
                               double *dx, PathState *st, const int *skip, double *resid,
                               unsigned long long limit_ns, int withhold = -1);
cudaError_t ph_mgs_cluster_launch(cudaStream_t stream, int C, int L, int N, int n, const double *A,
                                  long ldA, double *W, double *dx, PathState *st, const int *skip,
                                  double *resid, double *nrm_out);   // nrm_out: r_kk^2 (may be null)
