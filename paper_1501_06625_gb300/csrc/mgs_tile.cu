// mgs_tile.cu -- the least-squares solve of mgs.cu (MGS on the augmented
// matrix [J | rhs] and back substitution; Introduction, Section 3.1) for
// large shapes, as a tiled right-looking MGS with one grid barrier per pivot.
//
// The paper points to tiling (combining left- and right-looking MGS) to cut
// memory traffic on its GPU.  On GB300 the FP64 pipe is the bound and the
// whole matrix sits in L2, so what the tiling has to buy here is balance:
// the grid kernel of mgs.cu owns whole columns, and its slowest block carries
// ceil((n-k)/G) columns at pivot k.  Here the trailing matrix is cut into
// tiles of (row block) x (column group): G = R C blocks, block b takes row
// block r = b mod R (rows [r N / R, (r+1) N / R)) and the columns j = c mod C,
// c = b / R, so every block carries about N (n-k) / G (row, column) pairs.
//
// Per pivot k every block
//   1. waits at the grid barrier that closes pivot k-1;
//   2. sums the R partial dot products of every column it needs (written by
//      the R row blocks in the previous sweep): ||a_k||^2 (the pivot's norm,
//      whose reciprocal warp 0 computes) and a_k^H a_j for its own columns and
//      for column k+1, giving alpha_kj = a_k^H a_j / ||a_k||^2;
//   3. updates column k+1 for its own rows into shared memory (every block
//      of the row block does this redundantly: it needs those rows for the
//      next pivot's dot products, and recomputing them costs less than a
//      second barrier);
//   4. in one sweep over its tile: a_j -= alpha_kj a_k, then accumulates the
//      next pivot's partial dot product a_{k+1}^H a_j with the updated value
//      (for j = k+1 itself, ||a_{k+1}||^2), reduces it over the lanes of the
//      column and writes it for row block r;
//   5. arrives at the barrier.
// A sweep before pivot 0 only computes the partials of pivot 0; the sweep of
// pivot n-1 leaves the norm of the updated right-hand side, the least-squares
// residual.  Then block 0 solves the unit upper-triangular system in the
// alphas (dx_k = alpha_kn - sum_{j>k} alpha_kj dx_j), as mgs.cu does.
//
// Arithmetic is that of mgs.cu (unnormalised projections, q_k never formed,
// fused DD/QD dot-product and update terms); only the summation order of the
// dot products differs (R partial sums per column).  Matrix data written by
// another block is read through L2 only (ld.global.cg).  The barrier is a
// counter in the path state; every wait is bounded and a wait that runs out
// sets PathState::timeout.
#include "internal.h"
#include "mp.cuh"
#include "pathdev.cuh"

using namespace ph;

namespace {

constexpr int kTT = 256;                       // threads per block

PHD unsigned long long tile_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <class P>
PHD typename P::real ld_cg(const double *p, long stride, long i) {
  typename P::real z;
#pragma unroll
  for (int l = 0; l < P::L; ++l) P::set_limb(z, l, __ldcg(p + l * stride + i));
  return z;
}

template <class P>
PHD typename P::real ld_sh(const double *p, long stride, long i) {
  typename P::real z;
#pragma unroll
  for (int l = 0; l < P::L; ++l) P::set_limb(z, l, p[l * stride + i]);
  return z;
}

template <class P>
PHD void st_real(double *p, long stride, long i, const typename P::real &z) {
#pragma unroll
  for (int l = 0; l < P::L; ++l) p[l * stride + i] = P::limb(z, l);
}

template <class P>
__device__ typename P::real shfl_real(const typename P::real &a, int m) {
  typename P::real z;
#pragma unroll
  for (int l = 0; l < P::L; ++l) P::set_limb(z, l, __shfl_xor_sync(0xffffffffu, P::limb(a, l), m));
  return z;
}

template <class P>
__device__ typename P::real bcast_real(const typename P::real &a, int src) {
  typename P::real z;
#pragma unroll
  for (int l = 0; l < P::L; ++l) P::set_limb(z, l, __shfl_sync(0xffffffffu, P::limb(a, l), src));
  return z;
}

// Grid barrier: block arrivals counted in st->bar_count; waits for `target`.
// Returns false when the wait gave up (timeout flag set).
__device__ bool tile_barrier(PathState *st, unsigned target, unsigned long long limit_ns,
                             bool arrive = true) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (arrive) atomicAdd(&st->bar_count, 1u);
    volatile unsigned *cnt = &st->bar_count;
    volatile int *tmo = &st->timeout;
    int ok = 1;
    unsigned long long t0 = 0;
    unsigned spins = 0;
    while (*cnt < target) {
      if (*tmo) { ok = 0; break; }
      if ((++spins & 255u) == 0) {
        const unsigned long long now = tile_timer_ns();
        if (t0 == 0) t0 = now;
        else if (now - t0 > limit_ns) {
          atomicExch(&st->timeout, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Partials: part[parity][2L][R][nc], parity = (k+1) & 1 for the dot products
// against pivot k+1.  Shared memory: pv, nx: [2L][rows] the pivot rows and
// the updated rows of the next pivot column (the block's row block); y: [2L][n]
// (block 0, back substitution).
template <class P>
__global__ void __launch_bounds__(kTT, 1)
k_mgs_tile(int N, int n, int R, double *__restrict__ A, long ldA,
           double *__restrict__ W, double *__restrict__ nrm2, double *__restrict__ part,
           double *__restrict__ dx, PathState *st, const int *__restrict__ skip,
           double *__restrict__ resid, unsigned long long limit_ns, int withhold) {
  if (skip && *skip) return;
  typedef typename P::real real;
  typedef Part<P> PO;
  extern __shared__ double sm[];
  __shared__ real sh_inv, sh_dnr, sh_dni;
  __shared__ int sh_bad;
  bool bad = false;                                 // a zero or non-finite pivot: idle to the end
  const int nc = n + 1;
  const long Ap = (long)nc * ldA, Wp = (long)nc * nc;
  const int G = gridDim.x, C = G / R;
  const int b = blockIdx.x, r = b % R, c = b / R;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int rb = (int)(((long)r * N) / R), re = (int)(((long)(r + 1) * N) / R), rows = re - rb;
  const int rmax = (N + R - 1) / R;
  double *pv = sm, *nx = sm + 2L * P::L * rmax;
  const long PP = 2L * P::L * R * nc;              // doubles per parity
  int R2 = 1;
  while (R2 < R) R2 <<= 1;

  // the pivot "before pivot 0": nx = column 0 of the block's rows
  for (int u = tid; u < 2 * rows; u += kTT) {
    const int i = u >> 1, pt = u & 1;
#pragma unroll
    for (int l = 0; l < P::L; ++l)
      nx[(2 * l + pt) * rmax + i] = __ldcg(A + (2 * l + pt) * Ap + (rb + i));
  }
  __syncthreads();

  for (int k = -1; k < n; ++k) {
    const double *Ppar = part + (long)(k & 1) * PP;       // partials against pivot k
    double *Pnext = part + (long)((k + 1) & 1) * PP;      // partials against pivot k+1
    if (k >= 0) {
      if (!tile_barrier(st, (unsigned)G * (unsigned)(k + 1), limit_ns, !(b == 0 && k == withhold)))
        return;
      if (bad) continue;
      if (tid == 0) sh_bad = 0;
      // 2. ||a_k||^2 (warp 0) and a_k^H a_{k+1} (warp 1), summed over the R row blocks
      if (w == 0) {
        real s = P::zero();
        for (int q = lane; q < R; q += 32) s = P::add(s, ld_cg<P>(Ppar, (long)2 * R * nc, (long)q * nc + k));
        for (int m = (R2 < 32 ? R2 : 32) >> 1; m > 0; m >>= 1) s = P::add(s, shfl_real<P>(s, m));
        if (lane == 0) {
          const double lead = P::lead(s);
          if (!(lead > 0.0) || !isfinite(lead)) {
            sh_bad = 1;
            if (b == 0) atomicExch(&st->mgs_status, PH_NONFINITE);
          } else {
            sh_inv = P::recip(s);
            if (b == 0) st_real<P>(nrm2, nc, k, s);
          }
        }
      } else if (w == 1) {
        real sr = P::zero(), si = P::zero();
        for (int q = lane; q < R; q += 32) {
          sr = P::add(sr, ld_cg<P>(Ppar, (long)2 * R * nc, (long)q * nc + k + 1));
          si = P::add(si, ld_cg<P>(Ppar + (long)R * nc, (long)2 * R * nc, (long)q * nc + k + 1));
        }
        for (int m = (R2 < 32 ? R2 : 32) >> 1; m > 0; m >>= 1) {
          sr = P::add(sr, shfl_real<P>(sr, m));
          si = P::add(si, shfl_real<P>(si, m));
        }
        if (lane == 0) {
          sh_dnr = sr;
          sh_dni = si;
        }
      }
      __syncthreads();
      if (sh_bad) {                                 // the same decision in every block
        bad = true;
        continue;
      }
      // 3. column k+1 for this row block: nx = a_{k+1} - alpha_{k,k+1} a_k, with
      //    the pivot rows a_k (the previous nx) moved to pv
      const real inv = sh_inv;
      double *t = pv;
      pv = nx;
      nx = t;
      const real alr = P::mul(sh_dnr, inv), ali = P::mul(sh_dni, inv);
      if (b == 0 && tid == 0) {
#pragma unroll
        for (int l = 0; l < P::L; ++l) {
          W[(2 * l) * Wp + (long)(k + 1) * nc + k] = P::limb(alr, l);
          W[(2 * l + 1) * Wp + (long)(k + 1) * nc + k] = P::limb(ali, l);
        }
      }
      for (int u = tid; u < 2 * rows; u += kTT) {
        const int i = u >> 1, pt = u & 1;
        const double *ak1 = A + (long)(k + 1) * ldA + rb + i;
        const real ajr = ld_cg<P>(ak1, 2 * Ap, 0), aji = ld_cg<P>(ak1 + Ap, 2 * Ap, 0);
        const real akr = ld_sh<P>(pv + i, 2 * rmax, 0), aki = ld_sh<P>(pv + rmax + i, 2 * rmax, 0);
        const real v = pt == 0 ? PO::upd(ajr, alr, akr, ali, aki, 1.0)
                               : PO::upd(aji, alr, aki, ali, akr, -1.0);
#pragma unroll
        for (int l = 0; l < P::L; ++l) nx[(2 * l + pt) * rmax + i] = P::limb(v, l);
      }
      __syncthreads();
    }
    // 4. the sweep over the tile: columns j > k of group c.  Column k+1 (the
    //    next pivot) is not stored back: its updated rows live in nx, and no
    //    block reads it from A again (nor any column during the pivot it is
    //    the next pivot of), so the pre-pass of another block never sees it
    //    half updated.
    const int j0 = (k + 1) + ((c - (k + 1)) % C + C) % C;
    const int m = j0 <= n ? (n - j0) / C + 1 : 0;
    int S = 32;
    while (S > 1 && (long)m * S > kTT) S >>= 1;
    while (S > 1 && (S >> 1) >= rows) S >>= 1;     // no more lanes than rows
    const int slots = kTT / S, slot = tid / S, sl = tid % S;
    const int lead_lane = lane & ~(S - 1);          // first lane of this slot in the warp
    const real inv = k >= 0 ? sh_inv : P::zero();
    for (int q0 = 0; q0 < m; q0 += slots) {
      const int q = q0 + slot;
      const bool live = q < m;
      const int j = live ? j0 + q * C : n;
      const bool upd = live && k >= 0 && j > k + 1;
      // alpha_kj: the R partials of column j against pivot k, summed by the
      // lanes of the slot (every lane of the warp takes part in the shuffles)
      real alr = P::zero(), ali = P::zero();
      if (k >= 0) {
        real dr = P::zero(), di = P::zero();
        if (upd)
          for (int qq = sl; qq < R; qq += S) {
            dr = P::add(dr, ld_cg<P>(Ppar, (long)2 * R * nc, (long)qq * nc + j));
            di = P::add(di, ld_cg<P>(Ppar + (long)R * nc, (long)2 * R * nc, (long)qq * nc + j));
          }
        const int lim = R2 < S ? R2 : S;
        for (int mm = lim >> 1; mm > 0; mm >>= 1) {
          dr = P::add(dr, shfl_real<P>(dr, mm));
          di = P::add(di, shfl_real<P>(di, mm));
        }
        dr = bcast_real<P>(dr, lead_lane);
        di = bcast_real<P>(di, lead_lane);
        alr = P::mul(dr, inv);
        ali = P::mul(di, inv);
        if (upd && r == 0 && sl == 0) {
#pragma unroll
          for (int l = 0; l < P::L; ++l) {
            W[(2 * l) * Wp + (long)j * nc + k] = P::limb(alr, l);
            W[(2 * l + 1) * Wp + (long)j * nc + k] = P::limb(ali, l);
          }
        }
      }
      typename PO::acc ar = PO::zero(), ai = PO::zero();
      if (live) {
        double *aj = A + (long)j * ldA + rb;
        for (int i = sl; i < rows; i += S) {
          const real nr = ld_sh<P>(nx + i, 2 * rmax, 0), ni = ld_sh<P>(nx + rmax + i, 2 * rmax, 0);
          if (j == k + 1) {
            PO::sq(ar, nr);
            PO::sq(ar, ni);
          } else {
            real ajr = ld_cg<P>(aj + i, 2 * Ap, 0), aji = ld_cg<P>(aj + Ap + i, 2 * Ap, 0);
            if (upd) {
              const real akr = ld_sh<P>(pv + i, 2 * rmax, 0), aki = ld_sh<P>(pv + rmax + i, 2 * rmax, 0);
              const real ur = PO::upd(ajr, alr, akr, ali, aki, 1.0);
              const real ui = PO::upd(aji, alr, aki, ali, akr, -1.0);
              ajr = ur;
              aji = ui;
              st_real<P>(aj + i, 2 * Ap, 0, ajr);
              st_real<P>(aj + Ap + i, 2 * Ap, 0, aji);
            }
            // conj(a_{k+1}) a_j:  re = nr ajr + ni aji,  im = nr aji - ni ajr
            PO::dot2(ar, nr, ajr, ni, aji, 1.0);
            PO::dot2(ai, nr, aji, ni, ajr, -1.0);
          }
        }
      }
      // reduce over the S lanes of the slot (aligned groups within a warp)
      for (int mm = S >> 1; mm > 0; mm >>= 1) {
        ar = PO::combine(ar, PO::shfl(ar, mm));
        ai = PO::combine(ai, PO::shfl(ai, mm));
      }
      if (live && sl == 0) {
        const real vr = PO::value(ar), vi = PO::value(ai);
        st_real<P>(Pnext, (long)2 * R * nc, (long)r * nc + j, vr);
        st_real<P>(Pnext + (long)R * nc, (long)2 * R * nc, (long)r * nc + j, vi);
      }
    }
  }
  // completion: the partials of "pivot n" (the residual's norm) are written;
  // block 0 waits for every block and solves R dx = Q^H rhs, the others leave
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    atomicAdd(&st->bar_count, 1u);
  }
  if (b != 0) return;
  if (tid == 0) {
    volatile unsigned *cnt = &st->bar_count;
    volatile int *tmo = &st->timeout;
    const unsigned target = (unsigned)G * (unsigned)(n + 1);
    unsigned long long t0 = 0;
    unsigned spins = 0;
    while (*cnt < target) {
      if (*tmo) break;
      if ((++spins & 255u) == 0) {
        const unsigned long long now = tile_timer_ns();
        if (t0 == 0) t0 = now;
        else if (now - t0 > limit_ns) {
          atomicExch(&st->timeout, 1);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  if (*(volatile int *)&st->timeout) return;
  __syncthreads();
  if (tid == 0) st->bar_count = 0;                // every other block has left
  if (*(volatile int *)&st->mgs_status != PH_OK) return;
  {
    const double *Pn = part + (long)(n & 1) * PP;
    if (w == 0) {
      real s = P::zero();
      for (int q = lane; q < R; q += 32) s = P::add(s, ld_cg<P>(Pn, (long)2 * R * nc, (long)q * nc + n));
      for (int mm = (R2 < 32 ? R2 : 32) >> 1; mm > 0; mm >>= 1) s = P::add(s, shfl_real<P>(s, mm));
      if (lane == 0) {
        st_real<P>(nrm2, nc, n, s);
        if (resid) *resid = __dsqrt_rn(fmax(P::lead(s), 0.0));
      }
    }
  }
  // back substitution on y = alpha_{., n}:  dx_k = y_k;  y_i -= alpha_ik dx_k (i < k)
  double *s_y = sm;                                // [2L][n], the tile buffers are done
  __syncthreads();
  const double *yc = W + (long)n * nc;
  for (int i = tid; i < n; i += kTT) c_store<P>(s_y, n, i, c_load_cg<P>(yc, Wp, i));
  __syncthreads();
  const int part2 = (w >> 2) & 1;                  // warps 0-3 real, 4-7 imaginary
  const int r0 = (w & 3) * 32 + lane;              // rows r0, r0 + 128, ...
  for (int k = n - 1; k >= 1; --k) {
    const real xr = ld_sh<P>(s_y + k, 2L * n, 0), xi = ld_sh<P>(s_y + n + k, 2L * n, 0);
    const double *Wk = W + (long)k * nc;
    for (int i = r0; i < k; i += 128) {
      const real wr = ld_cg<P>(Wk + i, 2 * Wp, 0), wi = ld_cg<P>(Wk + Wp + i, 2 * Wp, 0);
      if (part2 == 0) {
        const real y = ld_sh<P>(s_y + i, 2L * n, 0);
        st_real<P>(s_y + i, 2L * n, 0, PO::upd(y, wr, xr, wi, xi, 1.0));
      } else {
        const real y = ld_sh<P>(s_y + n + i, 2L * n, 0);
        st_real<P>(s_y + n + i, 2L * n, 0, PO::upd(y, wr, xi, wi, xr, -1.0));
      }
    }
    __syncthreads();
  }
  double mx = 0.0;
  for (int i = tid; i < n; i += kTT) {
    cx<P> v = c_load<P>(s_y, n, i);
    c_store<P>(dx, n, i, v);
    const double a = c_mag_lead<P>(v);
    if (!(a <= mx)) mx = a;
  }
  atomicMax(&st->dx_bits, (unsigned long long)__double_as_longlong(mx));
}

template <class P>
size_t tile_smem(int N, int n, int R) {
  const int rmax = (N + R - 1) / R;
  const size_t a = sizeof(double) * 2 * 2 * P::L * (size_t)rmax;
  const size_t y = sizeof(double) * 2 * P::L * (size_t)n;
  return a > y ? a : y;
}

template <class P>
cudaError_t launch_tile(int G, int R, cudaStream_t stream, int N, int n, double *A, long ldA,
                        double *W, double *nrm2, double *part, double *dx, PathState *st,
                        const int *skip, double *resid, unsigned long long limit_ns,
                        int withhold) {
  const size_t smem = tile_smem<P>(N, n, R);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_mgs_tile<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  void *args[] = {&N, &n, &R, &A, &ldA, &W, &nrm2, &part, &dx, &st, (void *)&skip,
                  &resid, &limit_ns, &withhold};
  return cudaLaunchCooperativeKernel((const void *)k_mgs_tile<P>, dim3(G), dim3(kTT), args, smem,
                                     stream);
}

}  // namespace

// Blocks of the tiled solve for R row blocks: R * floor(sm_count / R), or 0
// when R does not fit (more row blocks than SMs, or the tile rows exceed the
// shared memory of a block).
int ph_mgs_tile_grid(int sm_count, int L, int N, int n, int R) {
  if (R < 1 || R > sm_count || R > N) return 0;
  const size_t smem = L == 1 ? tile_smem<F64>(N, n, R) : L == 2 ? tile_smem<DD>(N, n, R)
                                                                : tile_smem<QD>(N, n, R);
  if (smem > 227 * 1024) return 0;
  return R * (sm_count / R);
}

// Doubles of the partial-sum buffer of the tiled solve.
long ph_mgs_tile_part(int L, int n, int R) { return 2L * 2 * L * (long)R * (n + 1); }

cudaError_t ph_mgs_tile_launch(int sm_count, cudaStream_t stream, int L, int N, int n, int R,
                               double *A, long ldA, double *W, double *nrm2, double *part,
                               double *dx, PathState *st, const int *skip, double *resid,
                               unsigned long long limit_ns, int withhold) {
  const int G = ph_mgs_tile_grid(sm_count, L, N, n, R);
  if (G < 1) return cudaErrorInvalidValue;
  if (L == 1)
    return launch_tile<F64>(G, R, stream, N, n, A, ldA, W, nrm2, part, dx, st, skip, resid, limit_ns,
                            withhold);
  if (L == 2)
    return launch_tile<DD>(G, R, stream, N, n, A, ldA, W, nrm2, part, dx, st, skip, resid, limit_ns,
                           withhold);
  return launch_tile<QD>(G, R, stream, N, n, A, ldA, W, nrm2, part, dx, st, skip, resid, limit_ns,
                         withhold);
}
