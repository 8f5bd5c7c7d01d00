// mgs.cu -- least squares J dx = rhs by modified Gram-Schmidt on the augmented
// matrix A = [J | rhs] and back substitution (Introduction: MGS rather than
// LU with partial pivoting; Section 3.1: GPU_Modified_Gram_Schmidt).
//
// One persistent kernel per solve, its blocks co-resident (cooperative launch)
// and separated by a grid barrier after each column step.  Columns are dealt
// to blocks round-robin; each block's 256 threads split the rows.  Step k:
//   every block reads ||a_k||^2 (computed one step ahead by the owner of
//   column k, right after that column's last update), and for each of its
//   columns j > k forms d = a_k^H a_j, stores r_kj = d / r_kk and updates
//   a_j -= (d / ||a_k||^2) a_k, which equals a_j - r_kj q_k without forming
//   q_k = a_k / r_kk (Q is not needed for the solve).
// Column n (the right-hand side) ends as the least-squares residual, and its
// R entries are Q^H rhs.  Block 0 then solves R dx = Q^H rhs from the bottom
// up and accumulates max |dx_i| for the corrector.
//
// Data written by another block of the running kernel (the pivot column,
// the norms, R) is read through L2 only, since L1 is not coherent across SMs;
// the leading dimension of A is a multiple of 32 doubles so no cache line
// holds two columns.
//
// The grid barrier waits on a generation counter with a time limit (2 s of
// %globaltimer); a wait that runs out sets PathState::timeout and every block
// returns, so the host gets PH_TIMEOUT and the context stays usable.
#include "internal.h"
#include "mp.cuh"

using namespace ph;

namespace {

constexpr int kThreads = 256;
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
PHD cx<P> warp_sum_c(cx<P> v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    cx<P> o;
#pragma unroll
    for (int l = 0; l < P::L; ++l) {
      P::set_limb(o.re, l, __shfl_down_sync(0xffffffffu, P::limb(v.re, l), off));
      P::set_limb(o.im, l, __shfl_down_sync(0xffffffffu, P::limb(v.im, l), off));
    }
    v = c_add<P>(v, o);
  }
  return v;
}

// sum over the block; every thread gets the result
template <class P>
__device__ cx<P> block_sum_c(cx<P> v) {
  __shared__ cx<P> sh[kThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum_c<P>(v);
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < kThreads / 32 ? sh[lane] : c_zero<P>();
    v = warp_sum_c<P>(v);
    if (lane == 0) sh[0] = v;
  }
  __syncthreads();
  v = sh[0];
  __syncthreads();
  return v;
}

template <class P>
__device__ typename P::real col_norm2(const double *A, long Ap, long ldA, int N, int j) {
  cx<P> acc = c_zero<P>();
  for (int i = threadIdx.x; i < N; i += kThreads) {
    cx<P> a = c_load<P>(A + (long)j * ldA, Ap, i);
    acc.re = P::add(acc.re, c_abs2<P>(a));
  }
  return block_sum_c<P>(acc).re;
}

template <class P>
__global__ void __launch_bounds__(kThreads) k_mgs(int N, int n, double *__restrict__ A, long ldA,
                                                  double *__restrict__ R, double *__restrict__ nrm2,
                                                  double *__restrict__ irkk, double *__restrict__ dx,
                                                  PathState *st, const int *__restrict__ skip,
                                                  double *__restrict__ resid) {
  if (skip && *skip) return;
  const int nc = n + 1;
  const long Ap = (long)nc * ldA, Rp = (long)nc * nc;
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  typedef typename P::real real;

  if (b == 0) {
    real s = col_norm2<P>(A, Ap, ldA, N, 0);
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
    real inv2 = P::div(P::from(1.0), r2);
    real rkk = P::sqrt(r2);
    real irk = P::div(P::from(1.0), rkk);
    if (b == k % G && tid == 0) {
      c_store<P>(R + (long)k * nc, Rp, k, cx<P>{rkk, P::zero()});
      r_store<P>(irkk, n, k, irk);
    }
    int j = k + 1 + (((b - (k + 1)) % G) + G) % G;
    for (; j <= n; j += G) {
      cx<P> d = c_zero<P>();
      for (int i = tid; i < N; i += kThreads)
        d = c_add<P>(d, c_conj_mul<P>(c_load_cg<P>(A + (long)k * ldA, Ap, i),
                                      c_load<P>(A + (long)j * ldA, Ap, i)));
      d = block_sum_c<P>(d);
      if (tid == 0) c_store<P>(R + (long)j * nc, Rp, k, c_mul_real<P>(d, irk));
      cx<P> alpha = c_mul_real<P>(d, inv2);
      for (int i = tid; i < N; i += kThreads) {
        cx<P> aj = c_load<P>(A + (long)j * ldA, Ap, i);
        cx<P> ak = c_load_cg<P>(A + (long)k * ldA, Ap, i);
        c_store<P>(A + (long)j * ldA, Ap, i, c_sub<P>(aj, c_mul<P>(alpha, ak)));
      }
      if (j == k + 1) {
        real s = col_norm2<P>(A, Ap, ldA, N, j);
        if (tid == 0) r_store<P>(nrm2, nc, j, s);
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
  // back substitution on y = column n of R, in place
  __shared__ cx<P> s_x;
  double *y = R + (long)n * nc;
  for (int k = n - 1; k >= 0; --k) {
    if (tid == 0) {
      cx<P> xk = c_mul_real<P>(c_load_cg<P>(y, Rp, k), r_load_cg<P>(irkk, n, k));
      c_store<P>(dx, n, k, xk);
      s_x = xk;
    }
    __syncthreads();
    cx<P> xk = s_x;
    for (int i = tid; i < k; i += kThreads) {
      cx<P> yi = c_load_cg<P>(y, Rp, i);
      c_store<P>(y, Rp, i, c_sub<P>(yi, c_mul<P>(c_load_cg<P>(R + (long)k * nc, Rp, i), xk)));
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += kThreads)
    atomicMax(&st->dx_bits, (unsigned long long)__double_as_longlong(c_mag_lead<P>(c_load<P>(dx, n, i))));
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
  double *R = ctx->R.as<double>(), *nrm2 = ctx->nrm2.as<double>(), *irkk = ctx->irkk.as<double>();
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(ph_mgs_grid(ctx, L, N, n));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (L == 2)
    return cudaLaunchKernelEx(&cfg, k_mgs<DD>, N, n, A, ldA, R, nrm2, irkk, dx, st, skip, resid);
  return cudaLaunchKernelEx(&cfg, k_mgs<QD>, N, n, A, ldA, R, nrm2, irkk, dx, st, skip, resid);
}
