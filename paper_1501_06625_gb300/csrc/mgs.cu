// mgs.cu -- least squares J dx = rhs by modified Gram-Schmidt on the augmented
// matrix A = [J | rhs] and back substitution (Introduction: MGS rather than
// LU with partial pivoting; Section 3.1: GPU_Modified_Gram_Schmidt).
//
// One persistent kernel per solve.  Its blocks are co-resident (cooperative
// launch) and meet at a grid barrier after every column step.  Each block is
// one "column group" of TPC = 32..128 threads (one warp per SM sub-partition,
// so the group that owns the next pivot never shares an FP64 unit with another
// group); columns are dealt to blocks round-robin and a group's threads split
// the rows.  On GB300 every FP64 instruction of a warp costs ~64 cycles, so the
// length of the chain of dependent FP64 instructions per column step is what
// bounds a single solve; the formulation below keeps that chain short:
//
//   step k:  every group with a column j > k forms the unnormalised projection
//            alpha_kj = (a_k^H a_j) / ||a_k||^2   and updates a_j -= alpha_kj a_k,
//            which equals a_j - r_kj q_k of textbook MGS without forming q_k;
//            the owner of column k+1 then computes ||a_{k+1}||^2 for step k+1.
//   ||a_k||^2 needs one reciprocal per pivot (no square root, no division).
//   The rows of R are r_kj = alpha_kj ||a_k||, so R dx = Q^H rhs becomes the
//   unit upper-triangular system  dx_k = alpha_kn - sum_{j>k} alpha_kj dx_j,
//   solved by block 0 with one complex multiply-add per step on its chain.
//   Column n (rhs) ends as the least-squares residual vector.
//
// Data written by another block of the running kernel (the pivot column, the
// norms, the alphas) is read through L2 only (ld.global.cg), since L1 is not
// coherent across SMs; the leading dimension of A is a multiple of 32 doubles
// so no cache line holds two columns.
//
// The grid barrier waits on a generation counter with a time limit (2 s of
// %globaltimer); a wait that runs out sets PathState::timeout and every block
// returns, so the host gets PH_TIMEOUT and the context stays usable.
#include "internal.h"
#include "mp.cuh"

using namespace ph;

namespace {

constexpr unsigned long long kBarrierLimitNs = 2000000000ull;

PHD unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ bool grid_sync(PathState *st) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int *gen = &st->bar_gen;
    volatile int *tmo = &st->timeout;
    unsigned int g0 = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&st->bar_count, 1u) == gridDim.x - 1) {
      atomicExch(&st->bar_count, 0u);
      __threadfence();
      atomicAdd(&st->bar_gen, 1u);
    } else {
      unsigned long long t0 = global_timer_ns();
      while (*gen == g0) {
        if (*tmo) { ok = 0; break; }
        if (global_timer_ns() - t0 > kBarrierLimitNs) {
          atomicExch(&st->timeout, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <class P>
PHD typename P::real shfl_xor_r(const typename P::real &a, int m) {
  typename P::real z;
#pragma unroll
  for (int l = 0; l < P::L; ++l) P::set_limb(z, l, __shfl_xor_sync(0xffffffffu, P::limb(a, l), m));
  return z;
}

// Sum over the block (one column group of TPC threads); every thread gets it.
template <class P, int TPC>
__device__ cx<P> group_sum_c(cx<P> v) {
  __shared__ cx<P> sh[TPC / 32];
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) {
    v.re = P::add(v.re, shfl_xor_r<P>(v.re, m));
    v.im = P::add(v.im, shfl_xor_r<P>(v.im, m));
  }
  if (TPC == 32) return v;
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  v = sh[0];
#pragma unroll
  for (int w = 1; w < TPC / 32; ++w) v = c_add<P>(v, sh[w]);
  __syncthreads();
  return v;
}

template <class P, int TPC>
__device__ typename P::real group_sum_r(typename P::real v) {
  __shared__ typename P::real sh[TPC / 32];
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v = P::add(v, shfl_xor_r<P>(v, m));
  if (TPC == 32) return v;
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  v = sh[0];
#pragma unroll
  for (int w = 1; w < TPC / 32; ++w) v = P::add(v, sh[w]);
  __syncthreads();
  return v;
}

template <class P, int TPC>
__device__ typename P::real col_norm2(const double *A, long Ap, long ldA, int N, int j) {
  typename P::real acc = P::zero();
  for (int i = threadIdx.x; i < N; i += TPC)
    acc = P::add(acc, c_abs2<P>(c_load<P>(A + (long)j * ldA, Ap, i)));
  return group_sum_r<P, TPC>(acc);
}

// W: the alphas, [2L][nc][nc] column-major (alpha_kj at j*nc + k);
// inv2: 1/||a_k||^2, [L][n]; nrm2: ||a_k||^2, [L][n+1].
template <class P, int TPC>
__global__ void __launch_bounds__(TPC) k_mgs(int N, int n, double *__restrict__ A, long ldA,
                                             double *__restrict__ W, double *__restrict__ nrm2,
                                             double *__restrict__ inv2s, double *__restrict__ dx,
                                             PathState *st, const int *__restrict__ skip,
                                             double *__restrict__ resid) {
  if (skip && *skip) return;
  typedef typename P::real real;
  extern __shared__ double s_y[];          // back substitution: [2L][n]
  const int nc = n + 1;
  const long Ap = (long)nc * ldA, Wp = (long)nc * nc;
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;

  if (b == 0) {
    real s = col_norm2<P, TPC>(A, Ap, ldA, N, 0);
    if (tid == 0) r_store<P>(nrm2, nc, 0, s);
  }
  if (!grid_sync(st)) return;

  int status = PH_OK;
  for (int k = 0; k < n; ++k) {
    real r2 = r_load_cg<P>(nrm2, nc, k);
    double lead = P::lead(r2);
    if (!(lead > 0.0) || !isfinite(lead)) {   // the same decision in every block
      status = PH_NONFINITE;
      break;
    }
    int j = k + 1 + (((b - (k + 1)) % G) + G) % G;
    if (j <= n || b == 0) {
      real inv2 = P::recip(r2);
      if (b == 0 && tid == 0) r_store<P>(inv2s, n, k, inv2);
      for (; j <= n; j += G) {
        cx<P> d = c_zero<P>();
        for (int i = tid; i < N; i += TPC)
          d = c_add<P>(d, c_conj_mul<P>(c_load_cg<P>(A + (long)k * ldA, Ap, i),
                                        c_load<P>(A + (long)j * ldA, Ap, i)));
        d = group_sum_c<P, TPC>(d);
        cx<P> alpha = c_mul_real<P>(d, inv2);
        if (tid == 0) c_store<P>(W + (long)j * nc, Wp, k, alpha);
        for (int i = tid; i < N; i += TPC) {
          cx<P> aj = c_load<P>(A + (long)j * ldA, Ap, i);
          cx<P> ak = c_load_cg<P>(A + (long)k * ldA, Ap, i);
          c_store<P>(A + (long)j * ldA, Ap, i, c_sub<P>(aj, c_mul<P>(alpha, ak)));
        }
        if (j == k + 1) {
          real s = col_norm2<P, TPC>(A, Ap, ldA, N, j);
          if (tid == 0) r_store<P>(nrm2, nc, j, s);
        }
      }
    }
    if (!grid_sync(st)) return;
  }
  if (b != 0) return;
  if (status != PH_OK) {
    if (tid == 0) st->mgs_status = status;
    return;
  }
  // least-squares residual ||a_n|| after the last projection
  if (tid == 0 && resid) *resid = __dsqrt_rn(P::lead(r_load_cg<P>(nrm2, nc, n)));
  // back substitution on y = alpha_{., n}:  dx_k = y_k;  y_i -= alpha_ik dx_k (i < k)
  const double *y0 = W + (long)n * nc;
  for (int i = tid; i < n; i += TPC) c_store<P>(s_y, n, i, c_load_cg<P>(y0, Wp, i));
  __syncthreads();
  for (int k = n - 1; k >= 0; --k) {
    cx<P> xk = c_load<P>(s_y, n, k);
    if (tid == 0) c_store<P>(dx, n, k, xk);
    for (int i = tid; i < k; i += TPC) {
      cx<P> yi = c_load<P>(s_y, n, i);
      c_store<P>(s_y, n, i, c_sub<P>(yi, c_mul<P>(c_load_cg<P>(W + (long)k * nc, Wp, i), xk)));
    }
    __syncthreads();
  }
  double m = 0.0;
  for (int i = tid; i < n; i += TPC) {
    double a = c_mag_lead<P>(c_load<P>(s_y, n, i));
    if (!(a <= m)) m = a;
  }
  atomicMax(&st->dx_bits, (unsigned long long)__double_as_longlong(m));
}

template <class P, int TPC>
cudaError_t launch_tpc(ph_ctx *ctx, int N, int n, double *A, long ldA, double *W, double *nrm2,
                       double *inv2, double *dx, PathState *st, const int *skip, double *resid) {
  const size_t smem = sizeof(double) * 2 * P::L * (size_t)n;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_mgs<P, TPC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  // cooperative launch: the driver guarantees that all blocks are resident
  void *args[] = {&N, &n, &A, &ldA, &W, &nrm2, &inv2, &dx, &st, (void *)&skip, &resid};
  return cudaLaunchCooperativeKernel((const void *)k_mgs<P, TPC>,
                                     dim3(ph_mgs_grid(ctx, P::L, N, n)), dim3(TPC), args, smem,
                                     ctx->stream);
}

template <class P>
cudaError_t launch_p(ph_ctx *ctx, int N, int n, double *A, long ldA, double *W, double *nrm2,
                     double *inv2, double *dx, PathState *st, const int *skip, double *resid) {
  if (N <= 32) return launch_tpc<P, 32>(ctx, N, n, A, ldA, W, nrm2, inv2, dx, st, skip, resid);
  if (N <= 64) return launch_tpc<P, 64>(ctx, N, n, A, ldA, W, nrm2, inv2, dx, st, skip, resid);
  return launch_tpc<P, 128>(ctx, N, n, A, ldA, W, nrm2, inv2, dx, st, skip, resid);
}

}  // namespace

int ph_mgs_grid(ph_ctx *ctx, int L, int N, int n) {
  (void)L;
  (void)N;
  int g = n + 1 < ctx->sm_count ? n + 1 : ctx->sm_count;
  return g < 1 ? 1 : g;
}

cudaError_t ph_mgs_launch(ph_ctx *ctx, int L, int N, int n, double *A, long ldA, double *dx,
                          PathState *st, const int *skip, double *resid) {
  const int nc = n + 1;
  cudaError_t e;
  if ((e = ctx->R.ensure(sizeof(double) * 2 * L * (size_t)nc * nc)) != cudaSuccess) return e;
  if ((e = ctx->nrm2.ensure(sizeof(double) * L * (size_t)nc)) != cudaSuccess) return e;
  if ((e = ctx->irkk.ensure(sizeof(double) * L * (size_t)n)) != cudaSuccess) return e;
  double *W = ctx->R.as<double>(), *nrm2 = ctx->nrm2.as<double>(), *inv2 = ctx->irkk.as<double>();
  if (L == 2) return launch_p<DD>(ctx, N, n, A, ldA, W, nrm2, inv2, dx, st, skip, resid);
  return launch_p<QD>(ctx, N, n, A, ldA, W, nrm2, inv2, dx, st, skip, resid);
}

// The same solve with every buffer supplied by the caller and the launch
// configuration given explicitly (no context, no allocation): used by the
// allocation-free entry point in noalloc.cu.
cudaError_t ph_mgs_launch_buffers(int sm_count, cudaStream_t stream, int L, int N, int n,
                                  double *A, long ldA, double *W, double *nrm2, double *inv2,
                                  double *dx, PathState *st, double *resid) {
  ph_ctx tmp;                       // carries the SM count and the stream only
  tmp.sm_count = sm_count;
  tmp.stream = stream;
  if (L == 2) return launch_p<DD>(&tmp, N, n, A, ldA, W, nrm2, inv2, dx, st, nullptr, resid);
  return launch_p<QD>(&tmp, N, n, A, ldA, W, nrm2, inv2, dx, st, nullptr, resid);
}
