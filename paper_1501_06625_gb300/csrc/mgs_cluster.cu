// mgs_cluster.cu -- the least-squares solve of mgs.cu (MGS on [J | rhs] and
// back substitution; Introduction and Section 3.1) for small systems, on one
// thread-block cluster.
//
// For a single small solve (n up to a few hundred in DD) the grid kernel of
// mgs.cu is bound by the hand-off of each pivot between blocks through L2
// (a fence, a flag, a poll and dependent L2 loads: several microseconds per
// pivot, against ~2.5 us of arithmetic on the critical path).  Here the whole
// augmented matrix lives in the shared memory of the CTAs of one cluster:
// column j in CTA j mod C.  Per pivot k, a hardware cluster barrier makes the
// owner's finished column k and its norm visible; every CTA copies column k
// from the owner's shared memory (distributed shared memory) and updates its
// own columns j > k in place.  Pivot hand-off costs one cluster barrier.
//
// Arithmetic per column, as in mgs.cu: alpha_kj = (a_k^H a_j) / ||a_k||^2,
// a_j -= alpha_kj a_k (q_k never formed); R dx = Q^H rhs becomes
// dx_k = alpha_kn - sum_{j>k} alpha_kj dx_j.  The pivot's norm is not handed
// over: every pair of warps computes ||a_k||^2 from its copy of a_k together
// with its first dot product (two interleaved reductions), so the dependent
// chain between two pivots is one reduction, one reciprocal and one update.
//
// A pair of warps works on one column (one warp per real/imaginary part, a
// lane per row and its multiples of 32), synchronised by a named barrier.
// No CTA leaves before the end and no branch depends on computed values:
// every CTA passes the same cluster barriers and both warps of a pair the same
// named barriers, so no barrier can wait forever.
#include <cooperative_groups.h>

#include <type_traits>

#include "exsum.cuh"

#include "internal.h"
#include "mp.cuh"
#include "pathdev.cuh"

namespace cg = cooperative_groups;
using namespace ph;

namespace {

constexpr int kCT = 256;                 // threads per CTA: 8 warps, 4 pairs
constexpr int kPairs = kCT / 64;

// layout of a CTA's dynamic shared memory (doubles)
struct ClLayout {
  long cols, piv, xch, y, total;
};

__host__ __device__ inline ClLayout cl_layout(int L, int N, int n, int C) {
  const int cpc = (n + 1 + C - 1) / C;
  ClLayout o;
  o.cols = 0;                                        // [cpc][2L][N]
  o.piv = o.cols + (long)cpc * 2 * L * N;            // [2L][N] copy of the pivot column
  o.xch = o.piv + 2L * L * N;                        // [pairs][2 parts][2][L] exchange
  o.y = o.xch + (long)kPairs * 4 * L;                // [2L][n] back substitution (rank 0)
  o.total = o.y + 2L * L * n;
  return o;
}

__device__ __forceinline__ void pair_sync(int pair) {
  asm volatile("bar.sync %0, 64;" ::"r"(pair + 1) : "memory");
}

// the sum over the warp: exact integer sums for double-double and
// quad-double (exsum.cuh), a shuffle tree for one-limb types
template <class P>
__device__ typename P::real warp_total(typename Part<P>::acc a) {
  if constexpr (std::is_same<P, DD>::value || std::is_same<P, QD>::value) {
    return warp_exact_sum(Part<P>::value(a));
  } else {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) a = Part<P>::combine(a, Part<P>::shfl(a, m));
    return Part<P>::value(a);
  }
}

// two sums at once (independent chains, interleaved for one-limb types)
template <class P>
__device__ void warp_total2(typename Part<P>::acc a, typename Part<P>::acc b,
                            typename P::real &ra, typename P::real &rb) {
  if constexpr (std::is_same<P, DD>::value || std::is_same<P, QD>::value) {
    ra = warp_exact_sum(Part<P>::value(a));
    rb = warp_exact_sum(Part<P>::value(b));
  } else {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) {
      a = Part<P>::combine(a, Part<P>::shfl(a, m));
      b = Part<P>::combine(b, Part<P>::shfl(b, m));
    }
    ra = Part<P>::value(a);
    rb = Part<P>::value(b);
  }
}

// element (limb l, part c, row i) of a column block [2L][N]
template <class P>
__device__ __forceinline__ typename P::real col_part(const double *col, int N, int c, int i) {
  typename P::real z;
#pragma unroll
  for (int l = 0; l < P::L; ++l) P::set_limb(z, l, col[(2 * l + c) * N + i]);
  return z;
}

template <class P>
__device__ __forceinline__ void col_part_store(double *col, int N, int c, int i,
                                               const typename P::real &z) {
#pragma unroll
  for (int l = 0; l < P::L; ++l) col[(2 * l + c) * N + i] = P::limb(z, l);
}

template <class P>
__global__ void __launch_bounds__(kCT) k_mgs_cl(int N, int n, const double *__restrict__ A,
                                                long ldA, double *__restrict__ W,
                                                double *__restrict__ dx, PathState *st,
                                                const int *__restrict__ skip,
                                                double *__restrict__ resid,
                                                double *__restrict__ nrm_out) {
  if (skip && *skip) return;                       // the same value in every CTA
  typedef typename P::real real;
  typedef Part<P> PO;
  extern __shared__ double sm[];
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  const int nc = n + 1, cpc = (nc + C - 1) / C;
  const ClLayout o = cl_layout(P::L, N, n, C);
  double *cols = sm + o.cols, *piv = sm + o.piv, *xch = sm + o.xch;
  const long Ap = (long)nc * ldA, Wp = (long)nc * nc, csz = 2L * P::L * N;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int pair = w >> 1, part = w & 1;
  // this warp's exchange slots (dot part, norm part) and its partner's
  double *mine = xch + (4 * pair + 2 * part) * P::L;
  const double *other = xch + (4 * pair + 2 * (1 - part)) * P::L;

  // own columns into shared memory
  for (int s = 0; s < cpc; ++s) {
    const int j = rank + C * s;
    if (j > n) break;
    for (long e = tid; e < csz; e += kCT) {
      const long pl = e / N, i = e - pl * N;       // plane (2l + c), row
      cols[s * csz + e] = A[pl * Ap + (long)j * ldA + i];
    }
  }
  __syncthreads();

  // The control flow below depends on k, n, C, rank and pair only, never on
  // computed values: every CTA passes the same cluster barriers and both warps
  // of a pair the same named barriers.  A zero or non-finite pivot norm is
  // reported through st->mgs_status and the (meaningless) arithmetic goes on.
  for (int k = 0; k < n; ++k) {
    cl.sync();                                     // column k is final
    const double *rpiv = cl.map_shared_rank(cols + (k / C) * csz, k % C);
    for (long e = tid; e < csz; e += kCT) piv[e] = rpiv[e];
    __syncthreads();
    // this pair's columns j > k, the smallest (possibly the next pivot) first;
    // ||a_k||^2 is computed by each pair from its copy of a_k, alongside its
    // first dot product, so that no norm waits on the pivot's owner
    const int s0 = (k + 1 - rank + C - 1) / C;     // first slot with rank + C s > k
    real inv2 = P::zero(), r2 = P::zero();
    bool first = true;
    for (int s = s0 + pair; s < cpc; s += kPairs) {
      const int j = rank + C * s;
      if (j > n) break;
      double *cj = cols + s * csz;
      typename PO::acc a = PO::zero(), q = PO::zero();
      for (int i = lane; i < N; i += 32) {
        const real kr = col_part<P>(piv, N, 0, i), ki = col_part<P>(piv, N, 1, i);
        const real jr = col_part<P>(cj, N, 0, i), ji = col_part<P>(cj, N, 1, i);
        if (part == 0) PO::dot2(a, kr, jr, ki, ji, 1.0);
        else PO::dot2(a, kr, ji, ki, jr, -1.0);
        if (first) PO::sq(q, part == 0 ? kr : ki);
      }
      real d, nq;
      if (first) warp_total2<P>(a, q, d, nq);
      else d = warp_total<P>(a);
      if (lane == 0) {
        r_store<P>(mine, 1, 0, d);
        if (first) r_store<P>(mine + P::L, 1, 0, nq);
      }
      pair_sync(pair);
      const real d_o = r_load<P>(other, 1, 0);
      if (first) {
        const real nq_o = r_load<P>(other + P::L, 1, 0);
        r2 = part == 0 ? P::add(nq, nq_o) : P::add(nq_o, nq);     // the same in both warps
        inv2 = P::recip(r2);
        // a zero or non-finite pivot: reported by every pair that sees it (the
        // pair holding column n always does)
        if (part == 0 && lane == 0 && (!(P::lead(r2) > 0.0) || !isfinite(P::lead(r2))))
          atomicExch(&st->mgs_status, PH_NONFINITE);
        // ||a_k||^2 = r_kk^2 (leading limb), by the pair that holds column k+1
        if (nrm_out && j == k + 1 && part == 0 && lane == 0) nrm_out[k] = P::lead(r2);
      }
      pair_sync(pair);
      first = false;
      const real dr = part == 0 ? d : d_o, di = part == 0 ? d_o : d;
      const real alr = P::mul(dr, inv2), ali = P::mul(di, inv2);
      if (part == 0 && lane == 0) {
#pragma unroll
        for (int l = 0; l < P::L; ++l) {
          W[(2 * l) * Wp + (long)j * nc + k] = P::limb(alr, l);
          W[(2 * l + 1) * Wp + (long)j * nc + k] = P::limb(ali, l);
        }
      }
      // a_j -= alpha a_k:  re: jr - alr kr + ali ki;  im: ji - alr ki - ali kr
      for (int i = lane; i < N; i += 32) {
        const real kr = col_part<P>(piv, N, 0, i), ki = col_part<P>(piv, N, 1, i);
        if (part == 0)
          col_part_store<P>(cj, N, 0, i, PO::upd(col_part<P>(cj, N, 0, i), alr, kr, ali, ki, 1.0));
        else
          col_part_store<P>(cj, N, 1, i, PO::upd(col_part<P>(cj, N, 1, i), alr, ki, ali, kr, -1.0));
      }
    }
    __syncthreads();
  }
  cl.sync();                                       // every alpha written, column n final

  // the least-squares residual ||a_n||, by pair 0 of the owner of column n
  if (rank == n % C && pair == 0) {
    const double *cn = cols + (n / C) * csz;
    typename PO::acc q = PO::zero();
    for (int i = lane; i < N; i += 32) PO::sq(q, col_part<P>(cn, N, part, i));
    const real nq = warp_total<P>(q);
    if (lane == 0) r_store<P>(mine, 1, 0, nq);
    pair_sync(0);
    const real nq_o = r_load<P>(other, 1, 0);
    if (part == 0 && lane == 0 && resid) *resid = __dsqrt_rn(P::lead(P::add(nq, nq_o)));
  }
  if (rank != 0) return;
  __syncthreads();
  if (*(volatile int *)&st->mgs_status != PH_OK) return;
  // back substitution on y = alpha_{., n}:  dx_k = y_k;  y_i -= alpha_ik dx_k (i < k)
  double *y = sm + o.y;
  const double *yc = W + (long)n * nc;
  for (int i = tid; i < n; i += kCT) c_store<P>(y, n, i, c_load<P>(yc, Wp, i));
  __syncthreads();
  for (int k = n - 1; k >= 1; --k) {
    const real xr = r_load<P>(y, 2 * n, k), xi = r_load<P>(y + n, 2 * n, k);
    const double *Wk = W + (long)k * nc;
    for (int i = tid; i < 2 * k; i += kCT) {
      const int row = i >> 1, c = i & 1;           // (row, part) pairs
      const real wr = r_load<P>(Wk, 2 * Wp, row), wi = r_load<P>(Wk + Wp, 2 * Wp, row);
      const real yv = r_load<P>(y + c * n, 2 * n, row);
      const real nv = c == 0 ? PO::upd(yv, wr, xr, wi, xi, 1.0) : PO::upd(yv, wr, xi, wi, xr, -1.0);
      r_store<P>(y + c * n, 2 * n, row, nv);
    }
    __syncthreads();
  }
  double m = 0.0;
  for (int i = tid; i < n; i += kCT) {
    cx<P> v = c_load<P>(y, n, i);
    c_store<P>(dx, n, i, v);
    double a = c_mag_lead<P>(v);
    if (!(a <= m)) m = a;
  }
  atomicMax(&st->dx_bits, (unsigned long long)__double_as_longlong(m));
}

template <class P>
cudaError_t launch_cl(cudaStream_t stream, int C, int N, int n, const double *A, long ldA,
                      double *W, double *dx, PathState *st, const int *skip, double *resid,
                      double *nrm_out) {
  const size_t smem = sizeof(double) * (size_t)cl_layout(P::L, N, n, C).total;
  cudaError_t e = cudaFuncSetAttribute(k_mgs_cl<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(k_mgs_cl<P>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C);
  cfg.blockDim = dim3(kCT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_mgs_cl<P>, N, n, A, ldA, W, dx, st, skip, resid, nrm_out);
}

template <class P>
int max_cluster(int N, int n) {
  for (int C : {16, 8}) {
    const size_t smem = sizeof(double) * (size_t)cl_layout(P::L, N, n, C).total;
    if (smem > 227 * 1024) continue;
    if (cudaFuncSetAttribute(k_mgs_cl<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess ||
        (C > 8 && cudaFuncSetAttribute(k_mgs_cl<P>,
                                       cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                      cudaSuccess)) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(kCT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, k_mgs_cl<P>, &cfg) == cudaSuccess &&
        nclusters >= 1)
      return C;
    cudaGetLastError();
  }
  return 0;
}

}  // namespace

// The cluster size the cluster solve would use for this shape (16 or 8), or 0
// when the matrix does not fit in the shared memory of a cluster.
int ph_mgs_cluster_size(int L, int N, int n) {
  return L == 1 ? max_cluster<F64>(N, n) : L == 2 ? max_cluster<DD>(N, n) : max_cluster<QD>(N, n);
}

cudaError_t ph_mgs_cluster_launch(cudaStream_t stream, int C, int L, int N, int n, const double *A,
                                  long ldA, double *W, double *dx, PathState *st, const int *skip,
                                  double *resid, double *nrm_out) {
  if (L == 1) return launch_cl<F64>(stream, C, N, n, A, ldA, W, dx, st, skip, resid, nrm_out);
  if (L == 2) return launch_cl<DD>(stream, C, N, n, A, ldA, W, dx, st, skip, resid, nrm_out);
  return launch_cl<QD>(stream, C, N, n, A, ldA, W, dx, st, skip, resid, nrm_out);
}
