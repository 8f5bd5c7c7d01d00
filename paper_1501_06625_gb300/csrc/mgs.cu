// mgs.cu -- least squares J dx = rhs by modified Gram-Schmidt on the augmented
// matrix A = [J | rhs] and back substitution (Introduction: MGS rather than
// LU with partial pivoting; Section 3.1: GPU_Modified_Gram_Schmidt).
//
// One persistent kernel per solve, its blocks co-resident (cooperative launch).
// Columns are dealt to blocks round-robin; every block owns at least one.
// On GB300 an FP64 warp instruction occupies its SM sub-partition for ~64
// cycles whether or not the next one depends on it, so a single solve is
// bounded by the chain of FP64 instructions between one pivot and the next.
// The kernel is organised to keep that chain short:
//
//  * Unnormalised projections: for pivot k, each block forms
//      alpha_kj = (a_k^H a_j) / ||a_k||^2   and   a_j -= alpha_kj a_k   (j > k),
//    which equals a_j - r_kj q_k of textbook MGS without forming q_k.  The owner
//    of column k+1 updates that column first, computes ||a_{k+1}||^2 and
//    publishes the pivot (column + norm) through a per-column flag.  Blocks
//    wait only for the pivot they need (no grid barrier per step), and a block
//    whose columns are all done leaves.  One reciprocal per pivot; no square
//    root, no division.
//  * Each block has four warps, one per SM sub-partition: warps 0/1 carry the
//    real parts of two halves of the rows, warps 2/3 the imaginary parts, so a
//    complex dot product, update or norm costs each warp about half the FP64
//    instructions of the complex operation.
//  * Double-double reductions keep unnormalised (sum, compensation) pairs
//    through the tree (8 instructions per level instead of 11).
//  * R is never formed: with r_kj = alpha_kj ||a_k||, R dx = Q^H rhs becomes the
//    unit upper-triangular system dx_k = alpha_kn - sum_{j>k} alpha_kj dx_j,
//    solved by block 0 with one fused multiply-subtract per step on its chain.
//    Column n (rhs) ends as the least-squares residual vector.
//
// Data another block may have written (the pivot column, the norms, the
// alphas) is read through L2 only (ld.global.cg): L1 is not coherent across
// SMs.  The leading dimension of A is a multiple of 32 doubles so no cache line
// holds two columns.  Flags carry the solve's epoch (PathState::mgs_epoch + 1),
// so they need no clearing between the solves of one call.
//
// Every wait is bounded (2 s of %globaltimer); a wait that runs out sets
// PathState::timeout and the blocks return, so the host gets PH_TIMEOUT and the
// context stays usable.
#include <type_traits>

#include "exsum.cuh"
#include "internal.h"
#include "mp.cuh"
#include "pathdev.cuh"
#include "qfx.cuh"

using namespace ph;

namespace {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;   // default of the context setting
constexpr int kRowCache = 4;        // pivot rows a lane keeps in registers (N <= 128 WP)
constexpr int kDowndateBits = 20;   // cancellation beyond which a norm is recomputed
// Headroom (log2) of the QD fixed-point dot product over the bound ||a_k|| ||a_j||:
// one bit for rounding, the rest keeps every product's shift non-negative.
constexpr int kQfDotLg = 6;
// QD: the pivot column in fixed point in shared memory ([2][N] QF, aliasing the
// back substitution's buffer) up to this height
constexpr int kQfCacheMaxN = 2560;

PHD unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Thread 0 waits until *flag == tag (or the timeout flag is set); the block
// then proceeds.  The flag is read with acquire semantics, so every read the
// block makes after the barrier sees what the publisher wrote before its
// release.  Returns false when the wait gave up.
__device__ bool wait_flag(const int *flag, int tag, PathState *st, unsigned long long limit_ns) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    volatile int *tmo = &st->timeout;
    int ok = 1;
    if (ld_acquire(flag) != tag) {
      unsigned long long t0 = global_timer_ns();
      unsigned spins = 0;
      while (ld_acquire(flag) != tag) {
        if (*tmo) { ok = 0; break; }
        if ((++spins & 255u) == 0 && global_timer_ns() - t0 > limit_ns) {
          atomicExch(&st->timeout, 1);
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// After a block barrier, thread 0 stores the flag with release semantics:
// everything the block wrote before the barrier is visible to a block that
// reads the flag with acquire semantics.
__device__ void publish(int *flag, int tag) {
  __syncthreads();
  if (threadIdx.x == 0)
    asm volatile("st.release.gpu.global.b32 [%0], %1;" : : "l"(flag), "r"(tag) : "memory");
}

// Sum over the block's warps of one part: warps [0, WP) carry part 0, [WP, 2 WP)
// part 1.  Returns this warp's part total (normalised) to every lane.
template <class P, int WP>
__device__ typename P::real part_total(typename Part<P>::acc a, typename Part<P>::acc *sh) {
  typedef Part<P> PO;
  if constexpr (std::is_same<P, DD>::value) {      // an exact integer sum over the warp
    const dd v = warp_exact_sum(PO::value(a));
    a.s = v.h;
    a.c = v.l;
  } else if constexpr (std::is_same<P, QD>::value) {
    a.v = warp_exact_sum(a.v);
  } else {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) a = PO::combine(a, PO::shfl(a, m));
  }
  const int w = threadIdx.x >> 5, w0 = w - w % WP;
  if ((threadIdx.x & 31) == 0) sh[w] = a;
  __syncthreads();
  typename PO::acc t = sh[w0];
#pragma unroll
  for (int q = 1; q < WP; ++q) t = PO::combine(t, sh[w0 + q]);
  __syncthreads();
  return PO::value(t);
}

// Exchange a part value between the two halves of the block: warps of part q
// receive the value the warps of part 1-q computed.
template <class P, int WP>
__device__ typename P::real swap_parts(const typename P::real &mine, typename P::real *sh) {
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0 && w % WP == 0) sh[w / WP] = mine;
  __syncthreads();
  typename P::real other = sh[1 - w / WP];
  __syncthreads();
  return other;
}

// The same for two values at once (one pair of barriers).
template <class P, int WP>
__device__ void swap_parts2(const typename P::real &m1, const typename P::real &m2,
                            typename P::real *sh1, typename P::real *sh2, typename P::real &o1,
                            typename P::real &o2) {
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0 && w % WP == 0) {
    sh1[w / WP] = m1;
    sh2[w / WP] = m2;
  }
  __syncthreads();
  o1 = sh1[1 - w / WP];
  o2 = sh2[1 - w / WP];
  __syncthreads();
}

template <class P>
PHD typename P::real load_part(const double *col, long Ap, int part, long i) {
  typename P::real z;
#pragma unroll
  for (int l = 0; l < P::L; ++l) P::set_limb(z, l, col[(2 * l + part) * Ap + i]);
  return z;
}

template <class P>
PHD typename P::real load_part_cg(const double *col, long Ap, int part, long i) {
  typename P::real z;
#pragma unroll
  for (int l = 0; l < P::L; ++l) P::set_limb(z, l, __ldcg(col + (2 * l + part) * Ap + i));
  return z;
}

template <class P>
PHD void store_part(double *col, long Ap, int part, long i, const typename P::real &z) {
#pragma unroll
  for (int l = 0; l < P::L; ++l) col[(2 * l + part) * Ap + i] = P::limb(z, l);
}

// ||a_j||^2 of a column (after its last update by this block)
template <class P, int WP>
__device__ typename P::real col_norm2(const double *col, long Ap, int N, int part, int r0,
                                      typename Part<P>::acc *sh, typename P::real *shr) {
  typename Part<P>::acc a = Part<P>::zero();
  for (int i = r0; i < N; i += 32 * WP) Part<P>::sq(a, load_part<P>(col, Ap, part, i));
  typename P::real mine = part_total<P, WP>(a, sh);
  typename P::real other = swap_parts<P, WP>(mine, shr);
  return P::add(mine, other);
}

// W: alpha_kj at W[(2l+c) Wp + j nc + k] (column j of the alphas);
// nrm2: [L][nc] ||a_j||^2, then [L][nc] 1/||a_j||^2; ready: [nc] pivot flags.
template <class P, int WP>
__global__ void __launch_bounds__(64 * WP) k_mgs(int N, int n, double *__restrict__ A, long ldA,
                                                  double *__restrict__ W, double *__restrict__ nrm2,
                                                  double *__restrict__ dx, int *__restrict__ ready,
                                                  PathState *st, const int *__restrict__ skip,
                                                  double *__restrict__ resid,
                                                  unsigned long long limit_ns, int withhold) {
  if (skip && *skip) return;
  typedef typename P::real real;
  typedef Part<P> PO;
  __shared__ typename PO::acc sh_acc[2 * WP];
  __shared__ real sh_r[2];
  __shared__ real sh_d[2];                       // DD: the dot products of the two parts
  __shared__ int sh_rec;
  __shared__ Q256 sh_q[2 * WP];                  // QD dot products: each warp's fixed-point sum
  __shared__ int sh_qb[2 * WP];                  // and whether it met a non-finite value
  constexpr bool kQD = std::is_same<P, QD>::value;
  const bool qcache = kQD && N <= kQfCacheMaxN;
  extern __shared__ double s_y[];                // back substitution: [L][2][n]
  const int nc = n + 1;
  const long Ap = (long)nc * ldA, Wp = (long)nc * nc;
  double *ninv = nrm2 + (long)P::L * nc;
  const int G = gridDim.x, b = blockIdx.x, tid = threadIdx.x;
  const int w = tid >> 5, lane = tid & 31;
  const int part = w / WP;                       // 0 = real, 1 = imaginary
  constexpr int RS = 32 * WP;                    // row stride of a lane
  const int r0 = (w % WP) * 32 + lane;           // rows r0, r0 + RS, ...
  const int tag = st->mgs_epoch + 1;
  const int last_own = b + ((n - b) / G) * G;    // largest column this block owns

  // the norms of this block's columns; column 0 first, published at once
  for (int j = b; j <= n; j += G) {
    real s = col_norm2<P, WP>(A + (long)j * ldA, Ap, N, part, r0, sh_acc, sh_r);
    if (tid == 0) {
      r_store<P>(nrm2, nc, j, s);
      if (j == 0) r_store<P>(ninv, nc, 0, P::recip(s));
    }
    if (j == 0 && withhold != 0) publish(&ready[0], tag);
  }
  for (int k = 0; k < last_own; ++k) {
    if (!wait_flag(&ready[k], tag, st, limit_ns)) break;
    // the pivot's norm, its inverse and this lane's first kRowCache rows of
    // the pivot column (kept in registers for every column's dot product and
    // update), all requested before any of them is used
    const double *ak = A + (long)k * ldA;
    const real r2 = r_load_cg<P>(nrm2, nc, k);
    const real inv2 = r_load_cg<P>(ninv, nc, k);
    real ck_r[kRowCache], ck_i[kRowCache];
#pragma unroll
    for (int q = 0; q < kRowCache; ++q) {
      const int i = r0 + RS * q;
      if (i < N) {
        ck_r[q] = load_part_cg<P>(ak, Ap, 0, i);
        ck_i[q] = load_part_cg<P>(ak, Ap, 1, i);
      }
    }
    // warp 1 also updates warp 0's rows of the next pivot's column (below):
    // their first pivot row
    real c0_r = P::zero(), c0_i = P::zero();
    if (w == 1 && lane < N) {
      c0_r = load_part_cg<P>(ak, Ap, 0, lane);
      c0_i = load_part_cg<P>(ak, Ap, 1, lane);
    }
    const double lead = P::lead(r2);
    if (!(lead > 0.0) || !isfinite(lead) || !isfinite(P::lead(inv2))) {
      if (tid == 0) atomicExch(&st->mgs_status, PH_NONFINITE);   // the same value in every block
      break;
    }
    // QD: every row of the pivot column converted to fixed point once per pivot
    // (both parts), for every column's dot product and update (a finite norm
    // means finite entries)
    QF *s_piv = reinterpret_cast<QF *>(s_y);
    if constexpr (kQD) {
      if (qcache) {
        for (int i = tid; i < N; i += 64 * WP) {
          bool bad = false;
          s_piv[i] = qf_from(load_part_cg<P>(ak, Ap, 0, i), &bad);
          s_piv[N + i] = qf_from(load_part_cg<P>(ak, Ap, 1, i), &bad);
        }
        __syncthreads();
      }
    }
    for (int j = k + 1 + (((b - (k + 1)) % G) + G) % G; j <= n; j += G) {
      double *aj = A + (long)j * ldA;
      // ||a_j||^2 before this update, read before the barriers of the reduction
      // below (thread 0 overwrites it after them)
      const real old = r_load<P>(nrm2, nc, j);
      // this warp's part of a_k^H a_j:  re = akr ajr + aki aji,  im = akr aji - aki ajr
      real d, d_other = P::zero();                 // this part's sum; the other part's (QD)
      if constexpr (kQD) {
        // QD: every product in 256-bit fixed point (qfx.cuh), summed exactly
        // over the block.  ||a_k|| ||a_j|| bounds the sum of the products'
        // magnitudes (Cauchy-Schwarz), so it sets the accumulator's scale.
        // ||a_j||^2 is this column's current norm (downdated) or, for tall
        // columns, its first one, which only decreases under projection.
        const int er = (int)dbl_ef(P::lead(r2)), eo = (int)dbl_ef(P::lead(old));
        Q256 acc = q_zero();
        bool bad = eo == 0x7ff;
        const bool zero = eo == 0;
        const int kb = (er + eo + 1) / 2 + 1;        // ||a_k|| ||a_j|| < 2^(kb - 1022)
        const int base = kb - 1022 + kQfDotLg + 1 - 255;
        if (!zero && !bad && qcache) {
          for (int i = r0; i < N; i += RS) {
            const real ajr = load_part<P>(aj, Ap, 0, i), aji = load_part<P>(aj, Ap, 1, i);
            if (part == 0) qf_dot2c(acc, s_piv[i], ajr, s_piv[N + i], aji, 1.0, base, &bad);
            else qf_dot2c(acc, s_piv[i], aji, s_piv[N + i], ajr, -1.0, base, &bad);
          }
#pragma unroll
          for (int m = 16; m > 0; m >>= 1) acc = fix_add<4>(acc, q_shfl_xor(acc, m));
        } else if (!zero && !bad) {
#pragma unroll
          for (int q = 0; q < kRowCache; ++q) {
            const int i = r0 + RS * q;
            if (i < N) {
              const real ajr = load_part<P>(aj, Ap, 0, i), aji = load_part<P>(aj, Ap, 1, i);
              if (part == 0) qf_dot2(acc, ck_r[q], ajr, ck_i[q], aji, 1.0, base, &bad);
              else qf_dot2(acc, ck_r[q], aji, ck_i[q], ajr, -1.0, base, &bad);
            }
          }
          for (int i = r0 + RS * kRowCache; i < N; i += RS) {
            const real akr = load_part_cg<P>(ak, Ap, 0, i), aki = load_part_cg<P>(ak, Ap, 1, i);
            const real ajr = load_part<P>(aj, Ap, 0, i), aji = load_part<P>(aj, Ap, 1, i);
            if (part == 0) qf_dot2(acc, akr, ajr, aki, aji, 1.0, base, &bad);
            else qf_dot2(acc, akr, aji, aki, ajr, -1.0, base, &bad);
          }
#pragma unroll
          for (int m = 16; m > 0; m >>= 1) acc = fix_add<4>(acc, q_shfl_xor(acc, m));
        }
        const bool wbad = __any_sync(0xffffffffu, bad);
        if (lane == 0) {
          sh_q[w] = acc;
          sh_qb[w] = wbad;
        }
        __syncthreads();
        Q256 sp[2] = {sh_q[0], sh_q[WP]};
        int anybad = 0;
#pragma unroll
        for (int q = 0; q < 2 * WP; ++q) anybad |= sh_qb[q];
#pragma unroll
        for (int q = 1; q < WP; ++q) {
          sp[0] = fix_add<4>(sp[0], sh_q[q]);
          sp[1] = fix_add<4>(sp[1], sh_q[WP + q]);
        }
        real v[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          if (anybad) v[r] = P::from(__longlong_as_double(0x7ff8000000000000ll));
          else if (zero) v[r] = P::zero();
          else fix_round4(sp[r], base, v[r].x);
        }
        d = v[part];
        d_other = v[1 - part];
      } else {
        typename PO::acc a = PO::zero();
#pragma unroll
        for (int q = 0; q < kRowCache; ++q) {
          const int i = r0 + RS * q;
          if (i < N) {
            real ajr = load_part<P>(aj, Ap, 0, i), aji = load_part<P>(aj, Ap, 1, i);
            if (part == 0) PO::dot2(a, ck_r[q], ajr, ck_i[q], aji, 1.0);
            else PO::dot2(a, ck_r[q], aji, ck_i[q], ajr, -1.0);
          }
        }
        for (int i = r0 + RS * kRowCache; i < N; i += RS) {
          real akr = load_part_cg<P>(ak, Ap, 0, i), aki = load_part_cg<P>(ak, Ap, 1, i);
          real ajr = load_part<P>(aj, Ap, 0, i), aji = load_part<P>(aj, Ap, 1, i);
          if (part == 0) PO::dot2(a, akr, ajr, aki, aji, 1.0);
          else PO::dot2(a, akr, aji, aki, ajr, -1.0);
        }
        d = part_total<P, WP>(a, sh_acc);
      }
      real al = P::mul(d, inv2);                  // this part of alpha_kj
      real al_o;                                   // the other part
      if constexpr (std::is_same<P, DD>::value)
        swap_parts2<P, WP>(al, d, sh_r, sh_d, al_o, d_other);   // and its dot product
      else
        al_o = swap_parts<P, WP>(al, sh_r);
      const real alr = part == 0 ? al : al_o, ali = part == 0 ? al_o : al;
      // the update a - alr b + sg ali c of one part: QD in fixed point, with
      // alpha converted once per column
      QF qalr, qali;
      bool abad = false;
      if constexpr (kQD) {
        qalr = qf_from(alr, &abad);
        qali = qf_from(ali, &abad);
      }
      auto upd = [&](const real &x, const real &bb, const real &cc, double sg) -> real {
        if constexpr (kQD) return qf_upd2(x, qalr, bb, qali, cc, sg, abad);
        else return PO::upd(x, alr, bb, ali, cc, sg);
      };
      if (tid == 0) {
#pragma unroll
        for (int l = 0; l < P::L; ++l) {
          W[(2 * l) * Wp + (long)j * nc + k] = P::limb(alr, l);
          W[(2 * l + 1) * Wp + (long)j * nc + k] = P::limb(ali, l);
        }
      }
      // The norm of a_j after the update follows from alpha alone: a_j - alpha
      // a_k is orthogonal to a_k, so ||a_j||^2 - |alpha|^2 ||a_k||^2.  Where the
      // difference cancels more than kDowndateBits leading bits, the norm is
      // recomputed from the updated column; that decision reaches every thread
      // through shared memory.  For the next pivot's column (on the critical
      // chain) warp 0 computes the norm and its inverse while the other warps
      // update the column, warp 1 taking warp 0's rows of the real part too; for
      // other columns every warp updates its own rows and warp 0 then downdates.
      // Tall columns (N > 256) downdate nothing: a column's norm is needed only
      // when it becomes the next pivot, and there it is summed afresh from the
      // updated column (a downdate per column and pivot costs warp 0 more than
      // one fresh sum per column, and a fresh sum has no cancellation).
      const bool crit = j == k + 1;
      const bool fresh = N > 64 * kRowCache;
      const bool split = crit && !fresh && WP == 2;
      bool updated = false;
      if constexpr (kQD) {
        if (qcache) {                              // the pivot rows from shared memory
          if (!(split && w == 0)) {
            for (int i = r0; i < N; i += RS) {
              if (part == 0)
                store_part<P>(aj, Ap, 0, i, qf_upd3(load_part<P>(aj, Ap, 0, i), qalr, s_piv[i], qali,
                                                    s_piv[N + i], 1.0, abad));
              else
                store_part<P>(aj, Ap, 1, i, qf_upd3(load_part<P>(aj, Ap, 1, i), qalr, s_piv[N + i],
                                                    qali, s_piv[i], -1.0, abad));
            }
            if (split && w == 1)                   // warp 0's rows of the real part
              for (int i = lane; i < N; i += 64)
                store_part<P>(aj, Ap, 0, i, qf_upd3(load_part<P>(aj, Ap, 0, i), qalr, s_piv[i], qali,
                                                    s_piv[N + i], 1.0, abad));
          }
          updated = true;
        }
      }
      if (!updated && !(split && w == 0)) {
        // a_j -= alpha a_k:  re: ajr - alr akr + ali aki;  im: aji - alr aki - ali akr
#pragma unroll
        for (int q = 0; q < kRowCache; ++q) {
          const int i = r0 + RS * q;
          if (i < N) {
            if (part == 0)
              store_part<P>(aj, Ap, 0, i,
                            upd(load_part<P>(aj, Ap, 0, i), ck_r[q], ck_i[q], 1.0));
            else
              store_part<P>(aj, Ap, 1, i,
                            upd(load_part<P>(aj, Ap, 1, i), ck_i[q], ck_r[q], -1.0));
          }
        }
        for (int i = r0 + RS * kRowCache; i < N; i += RS) {
          real akr = load_part_cg<P>(ak, Ap, 0, i), aki = load_part_cg<P>(ak, Ap, 1, i);
          if (part == 0)
            store_part<P>(aj, Ap, 0, i, upd(load_part<P>(aj, Ap, 0, i), akr, aki, 1.0));
          else
            store_part<P>(aj, Ap, 1, i, upd(load_part<P>(aj, Ap, 1, i), aki, akr, -1.0));
        }
        if (split && w == 1) {                     // warp 0's rows of the real part
          for (int i = lane; i < N; i += 64) {
            real akr = c0_r, aki = c0_i;
            if (i != lane) {
              akr = load_part_cg<P>(ak, Ap, 0, i);
              aki = load_part_cg<P>(ak, Ap, 1, i);
            }
            store_part<P>(aj, Ap, 0, i, upd(load_part<P>(aj, Ap, 0, i), akr, aki, 1.0));
          }
        }
      }
      if (fresh) {
        if (crit) {                                // the same branch in every thread
          __syncthreads();
          const real s = col_norm2<P, WP>(aj, Ap, N, part, r0, sh_acc, sh_r);
          if (tid == 0) {
            r_store<P>(nrm2, nc, j, s);
            r_store<P>(ninv, nc, j, P::recip(s));
          }
        }
      } else {
        if (w == 0) {
          real s;
          if constexpr (kQD) {
            // ||a_j||^2 - |alpha|^2 ||a_k||^2 = ||a_j||^2 - Re(d conj(alpha)), d
            // = a_k^H a_j (warp 0 carries the real part), in fixed point
            bool b2 = abad;
            const QF A = qf_from(old, &b2);
            const QF p1 = qf_mul(qf_from(d, &b2), qalr);
            const QF p2 = qf_mul(qf_from(d_other, &b2), qali);
            const QF t[3] = {A, qf_neg(p1), qf_neg(p2)};
            s = b2 ? P::from(__longlong_as_double(0x7ff8000000000000ll)) : qf_sum_to_qd<3>(t);
          } else if constexpr (std::is_same<P, DD>::value) {
            // |alpha|^2 ||a_k||^2 = Re(d conj(alpha)) = Re d Re alpha + Im d Im alpha
            // (warp 0 carries the real parts), one fused DD sum of two products:
            // 30 FP64 instructions on warp 0's chain where the DD products take 43
            dd t;
            cops<DD>::part(d.h, d.l, alr.h, alr.l, d_other.h, d_other.l, ali.h, ali.l, 1.0, t.h,
                           t.l);
            s = DD::sub(old, t);
          } else {
            s = P::sub(old, P::mul(P::add(P::mul(alr, alr), P::mul(ali, ali)), r2));
          }
          const bool rec = !(P::lead(s) > ldexp(P::lead(old), -kDowndateBits));
          if (lane == 0) {
            sh_rec = rec;
            if (!rec) {
              r_store<P>(nrm2, nc, j, s);
              if (crit) r_store<P>(ninv, nc, j, P::recip(s));
            }
          }
        }
        __syncthreads();
        if (sh_rec) {                              // the same value in every thread
          const real s = col_norm2<P, WP>(aj, Ap, N, part, r0, sh_acc, sh_r);
          if (tid == 0) {
            r_store<P>(nrm2, nc, j, s);
            if (j == k + 1) r_store<P>(ninv, nc, j, P::recip(s));
          }
        }
      }
      if (j == k + 1 && j != withhold) publish(&ready[j], tag);
    }
  }
  // completion: block 0 waits for every block, then solves R dx = Q^H rhs
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    atomicAdd(&st->mgs_done, 1u);
  }
  if (b != 0) return;
  if (tid == 0) {
    volatile unsigned int *done = &st->mgs_done;
    volatile int *tmo = &st->timeout;
    unsigned long long t0 = global_timer_ns();
    unsigned spins = 0;
    while (*done < (unsigned)G) {
      if (*tmo) break;
      if ((++spins & 255u) == 0 && global_timer_ns() - t0 > limit_ns) {
        atomicExch(&st->timeout, 1);
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  if (*(volatile int *)&st->timeout) return;
  __syncthreads();
  if (tid == 0) {
    st->mgs_done = 0;
    st->mgs_epoch = tag;                           // this solve's flags become stale
  }
  if (*(volatile int *)&st->mgs_status != PH_OK) return;
  if (tid == 0 && resid) *resid = __dsqrt_rn(P::lead(r_load_cg<P>(nrm2, nc, n)));
  // back substitution on y = alpha_{., n}:  dx_k = y_k;  y_i -= alpha_ik dx_k (i < k)
  const double *yc = W + (long)n * nc;
  for (int i = tid; i < n; i += 64 * WP) c_store<P>(s_y, n, i, c_load_cg<P>(yc, Wp, i));
  __syncthreads();
  for (int k = n - 1; k >= 1; --k) {
    const real xr = load_part<P>(s_y, n, 0, k), xi = load_part<P>(s_y, n, 1, k);
    const double *Wk = W + (long)k * nc;
    // warps of part 0 update the real parts of rows i < k, part 1 the imaginary
    for (int i = r0; i < k; i += RS) {
      real wr = load_part_cg<P>(Wk, Wp, 0, i), wi = load_part_cg<P>(Wk, Wp, 1, i);
      if (part == 0) store_part<P>(s_y, n, 0, i, PO::upd(load_part<P>(s_y, n, 0, i), wr, xr, wi, xi, 1.0));
      else store_part<P>(s_y, n, 1, i, PO::upd(load_part<P>(s_y, n, 1, i), wr, xi, wi, xr, -1.0));
    }
    __syncthreads();
  }
  double m = 0.0;
  for (int i = tid; i < n; i += 64 * WP) {
    cx<P> v = c_load<P>(s_y, n, i);
    c_store<P>(dx, n, i, v);
    double a = c_mag_lead<P>(v);
    if (!(a <= m)) m = a;
  }
  atomicMax(&st->dx_bits, (unsigned long long)__double_as_longlong(m));
}

template <class P, int WP>
cudaError_t launch_wp(int sm_count, cudaStream_t stream, int N, int n, double *A, long ldA,
                      double *W, double *nrm2, double *dx, int *ready, PathState *st,
                      const int *skip, double *resid, unsigned long long limit_ns, int withhold) {
  size_t smem = sizeof(double) * 2 * P::L * (size_t)n;
  if (std::is_same<P, QD>::value && N <= kQfCacheMaxN && sizeof(QF) * 2 * (size_t)N > smem)
    smem = sizeof(QF) * 2 * (size_t)N;            // the pivot column in fixed point
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_mgs<P, WP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  int grid = n + 1 < sm_count ? n + 1 : sm_count;
  if (grid < 1) grid = 1;
  // cooperative launch: the driver guarantees that all blocks are resident
  void *args[] = {&N, &n, &A, &ldA, &W, &nrm2, &dx, &ready, &st, (void *)&skip, &resid,
                  &limit_ns, &withhold};
  return cudaLaunchCooperativeKernel((const void *)k_mgs<P, WP>, dim3(grid), dim3(64 * WP), args,
                                     smem, stream);
}

// Two warps per part (128 threads); four (256 threads) for QD columns taller
// than 128 rows.  With FP64 sums four warps per part measured slower on tall
// QD matrices (259 against 235 ms at 512 x 513: the FP64 pipe was already
// full); with the fixed-point QD arithmetic the integer chains are
// latency-bound and twice the warps hide more of it (134 -> 107 ms at
// 512 x 513, 29.6 -> 26.3 ms at 256 x 257).
template <class P>
cudaError_t launch_p(int sm_count, cudaStream_t stream, int N, int n, double *A, long ldA,
                     double *W, double *nrm2, double *dx, int *ready, PathState *st,
                     const int *skip, double *resid, unsigned long long limit_ns = kWaitLimitNs,
                     int withhold = -1) {
  if (std::is_same<P, QD>::value && N > 128)
    return launch_wp<P, 4>(sm_count, stream, N, n, A, ldA, W, nrm2, dx, ready, st, skip, resid,
                           limit_ns, withhold);
  return launch_wp<P, 2>(sm_count, stream, N, n, A, ldA, W, nrm2, dx, ready, st, skip, resid,
                         limit_ns, withhold);
}

}  // namespace

int ph_mgs_grid(ph_ctx *ctx, int L, int N, int n) {
  (void)L;
  (void)N;
  int g = n + 1 < ctx->sm_count ? n + 1 : ctx->sm_count;
  return g < 1 ? 1 : g;
}

namespace {

// A diagonally dominant complex matrix in the leading limbs, for timing: the
// time of a solve depends on the shape, not on the values (beyond their being
// finite and the matrix nonsingular).
__global__ void k_tune_fill(double *A, int N, long ldA, long Ap, long total) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total;
       e += (long)gridDim.x * blockDim.x) {
    const long pl = e / Ap, r = e - pl * Ap;
    const long j = r / ldA, i = r - j * ldA;
    double v = 0.0;
    if (pl < 2 && i < N) {
      unsigned h = (unsigned)(i * 7919 + j * 104729 + pl * 31);
      h ^= h >> 13;
      h *= 0x5bd1e995u;
      h ^= h >> 15;
      v = ((double)(h & 0xffffu) / 65536.0 - 0.5) * 0.1;
      if (pl == 0 && i == j) v += 4.0;
    }
    A[e] = v;
  }
}

}  // namespace

long ph_lda(int N);
cudaError_t ph_mgs_launch_buffers(int sm_count, cudaStream_t stream, int L, int N, int n,
                                  double *A, long ldA, double *W, double *nrm2, double *dx,
                                  int *ready, PathState *st, double *resid);

// Variant codes (ph_ctx::mgs_variant): the kind times 4096 plus its size.
static int mgs_code(int kind, int size) { return kind * 4096 + size; }
static int mgs_kind(int code) { return code / 4096; }
static int mgs_size(int code) { return code % 4096; }
static long long mgs_key(int L, int N, int n) {
  return ((long long)L << 48) | ((long long)N << 24) | (long long)n;
}

// Row-block counts of the tiled kernel worth timing for a shape: powers of
// two with at least 8 rows per block that fit (ph_mgs_tile_grid).
static std::vector<int> tile_candidates(ph_ctx *ctx, int L, int N, int n) {
  std::vector<int> out;
  for (int R = 1; R <= 64; R *= 2)
    if ((R == 1 || N / R >= 8) && ph_mgs_tile_grid(ctx->sm_count, L, N, n, R) > 0) out.push_back(R);
  return out;
}

// Buffers a variant needs beyond A and dx (sized before any graph capture).
static cudaError_t mgs_buffers(ph_ctx *ctx, int L, int n, int code) {
  const int nc = n + 1;
  cudaError_t e;
  if ((e = ctx->R.ensure(sizeof(double) * 2 * L * (size_t)nc * nc)) != cudaSuccess) return e;
  if ((e = ctx->nrm2.ensure(sizeof(double) * 2 * L * (size_t)nc)) != cudaSuccess) return e;
  if ((e = ctx->flags.ensure(sizeof(int) * (size_t)nc)) != cudaSuccess) return e;
  if (mgs_kind(code) == PH_MGS_TILED)
    e = ctx->mgs_part.ensure(sizeof(double) * (size_t)ph_mgs_tile_part(L, n, mgs_size(code)));
  return e;
}

static cudaError_t mgs_launch_code(ph_ctx *ctx, int code, cudaStream_t s, int L, int N, int n,
                                   double *A, long ldA, double *W, double *nrm2, double *dx,
                                   int *flags, PathState *st, const int *skip, double *resid) {
  const int kind = mgs_kind(code), size = mgs_size(code);
  if (kind == PH_MGS_CLUSTER)
    return ph_mgs_cluster_launch(s, size, L, N, n, A, ldA, W, dx, st, skip, resid, nrm2);
  if (kind == PH_MGS_TILED)
    return ph_mgs_tile_launch(ctx->sm_count, s, L, N, n, size, A, ldA, W, nrm2,
                              ctx->mgs_part.as<double>(), dx, st, skip, resid, ctx->wait_ns,
                              ctx->withhold);
  if (L == 1)
    return launch_p<F64>(ctx->sm_count, s, N, n, A, ldA, W, nrm2, dx, flags, st, skip, resid,
                         ctx->wait_ns, ctx->withhold);
  if (L == 2)
    return launch_p<DD>(ctx->sm_count, s, N, n, A, ldA, W, nrm2, dx, flags, st, skip, resid,
                        ctx->wait_ns, ctx->withhold);
  return launch_p<QD>(ctx->sm_count, s, N, n, A, ldA, W, nrm2, dx, flags, st, skip, resid,
                      ctx->wait_ns, ctx->withhold);
}

// Times the variants of a shape once per context on a scratch matrix and
// keeps the fastest (the grid kernel, the cluster kernel where the matrix
// fits a cluster, the tiled kernel for each row-block count worth trying).
// Outside stream capture only; during a capture an unmeasured shape gets the
// grid kernel.  Returns the variant code.
int ph_mgs_tune(ph_ctx *ctx, int L, int N, int n) {
  const long long key = mgs_key(L, N, n);
  auto it = ctx->mgs_variant.find(key);
  if (it != ctx->mgs_variant.end()) return it->second;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(ctx->stream, &cs) != cudaSuccess ||
      cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return 0;
  }
  std::vector<int> codes = {mgs_code(PH_MGS_GRID, 0)};
  const int C = ph_mgs_cluster_size(L, N, n);
  cudaGetLastError();
  if (C > 0) codes.push_back(mgs_code(PH_MGS_CLUSTER, C));
  for (int R : tile_candidates(ctx, L, N, n)) codes.push_back(mgs_code(PH_MGS_TILED, R));
  const int nc = n + 1;
  const long ldA = ph_lda(N), Ap = (long)nc * ldA, total = 2L * L * Ap;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = ctx->tuneA.ensure(sizeof(double) * total);
  if (e == cudaSuccess) e = ctx->tuneW.ensure(sizeof(double) * 2 * L * (size_t)nc * nc);
  if (e == cudaSuccess) e = ctx->tuneN.ensure(sizeof(double) * 2 * L * (size_t)nc);
  if (e == cudaSuccess) e = ctx->tuneF.ensure(sizeof(int) * (size_t)nc);
  if (e == cudaSuccess) e = ctx->tuneX.ensure(sizeof(double) * 2 * L * (size_t)n);
  if (e == cudaSuccess) e = ctx->tuneS.ensure(sizeof(PathState));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  PathState *st = ctx->tuneS.as<PathState>();
  double *A = ctx->tuneA.as<double>();
  float best_all = 1e30f;
  int choice = 0;
  MgsTimes times;
  for (int code : codes) {
    if (e != cudaSuccess) break;
    if (mgs_kind(code) == PH_MGS_TILED &&
        (e = mgs_buffers(ctx, L, n, code)) != cudaSuccess)
      break;
    float best = 1e30f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {     // rep 0 warms up
      k_tune_fill<<<64, 256, 0, ctx->stream>>>(A, N, ldA, Ap, total);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaMemsetAsync(st, 0, sizeof(PathState), ctx->stream);
      if (e == cudaSuccess) e = cudaMemsetAsync(ctx->tuneF.p, 0, sizeof(int) * nc, ctx->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
      if (e == cudaSuccess)
        e = mgs_launch_code(ctx, code, ctx->stream, L, N, n, A, ldA, ctx->tuneW.as<double>(),
                            ctx->tuneN.as<double>(), ctx->tuneX.as<double>(),
                            ctx->tuneF.as<int>(), st, nullptr, nullptr);
      if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && rep > 0 && ms < best) best = ms;
      if (e == cudaSuccess && rep == 1 && ms > 50.0f) break;    // long solves: one timed run
    }
    if (e != cudaSuccess) break;
    const int kind = mgs_kind(code);
    if (best < times.ms[kind]) {
      times.ms[kind] = best;
      if (kind == PH_MGS_TILED) times.tile_R = mgs_size(code);
    }
    if (best < best_all) {
      best_all = best;
      choice = code;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    choice = 0;
  } else {
    ctx->mgs_times[key] = times;
  }
  if (mgs_buffers(ctx, L, n, choice) != cudaSuccess) {
    cudaGetLastError();
    choice = 0;
  }
  ctx->mgs_variant[key] = choice;
  return choice;
}

cudaError_t ph_mgs_launch(ph_ctx *ctx, int L, int N, int n, double *A, long ldA, double *dx,
                          PathState *st, const int *skip, double *resid) {
  const int code = ph_mgs_tune(ctx, L, N, n);
  cudaError_t e = mgs_buffers(ctx, L, n, code);
  if (e != cudaSuccess) return e;
  return mgs_launch_code(ctx, code, ctx->stream, L, N, n, A, ldA, ctx->R.as<double>(),
                         ctx->nrm2.as<double>(), dx, ctx->flags.as<int>(), st, skip, resid);
}

// The same solve with every buffer supplied by the caller and the launch
// configuration given explicitly (no context, no allocation): used by the
// allocation-free entry point in noalloc.cu.  `ready` holds n+1 ints that must
// not hold the value PathState::mgs_epoch + 1 (zeroed flags with a zeroed state
// qualify).
cudaError_t ph_mgs_launch_buffers(int sm_count, cudaStream_t stream, int L, int N, int n,
                                  double *A, long ldA, double *W, double *nrm2, double *dx,
                                  int *ready, PathState *st, double *resid) {
  if (L == 1)
    return launch_p<F64>(sm_count, stream, N, n, A, ldA, W, nrm2, dx, ready, st, nullptr, resid);
  if (L == 2)
    return launch_p<DD>(sm_count, stream, N, n, A, ldA, W, nrm2, dx, ready, st, nullptr, resid);
  return launch_p<QD>(sm_count, stream, N, n, A, ldA, W, nrm2, dx, ready, st, nullptr, resid);
}

extern "C" ph_status ph_mgs_variant(ph_ctx *ctx, ph_prec prec, int N, int n, int *kind, int *size,
                                    double *ms) {
  if (!ctx) return PH_EINVAL;
  const int L = (int)prec;
  if ((L != 1 && L != 2 && L != 4) || n < 1 || N < n || !kind || !size)
    return ph_fail(ctx, PH_EINVAL, "ph_mgs_variant: invalid argument");
  cudaSetDevice(ctx->device);
  const int code = ph_mgs_tune(ctx, L, N, n);
  *kind = mgs_kind(code);
  *size = mgs_size(code);
  if (ms) {
    auto it = ctx->mgs_times.find(mgs_key(L, N, n));
    for (int q = 0; q < 3; ++q)
      ms[q] = it != ctx->mgs_times.end() && it->second.ms[q] < 1e29f ? it->second.ms[q] : -1.0;
  }
  return PH_OK;
}

void ph_track_release(ph_ctx *ctx);

extern "C" ph_status ph_mgs_set_variant(ph_ctx *ctx, ph_prec prec, int N, int n, int kind,
                                        int size) {
  if (!ctx) return PH_EINVAL;
  const int L = (int)prec;
  if ((L != 1 && L != 2 && L != 4) || n < 1 || N < n || kind < -1 || kind > PH_MGS_TILED)
    return ph_fail(ctx, PH_EINVAL, "ph_mgs_set_variant: invalid argument");
  cudaSetDevice(ctx->device);
  const long long key = mgs_key(L, N, n);
  if (kind == PH_MGS_CLUSTER && (size < 1 || size != ph_mgs_cluster_size(L, N, n)))
    return ph_fail(ctx, PH_EINVAL, "ph_mgs_set_variant: the shape does not take that cluster size");
  if (kind == PH_MGS_TILED && ph_mgs_tile_grid(ctx->sm_count, L, N, n, size) < 1)
    return ph_fail(ctx, PH_EINVAL, "ph_mgs_set_variant: no tiled solve with that many row blocks");
  if (kind < 0) {
    ctx->mgs_variant.erase(key);
    ctx->mgs_times.erase(key);
  } else {
    const int code = mgs_code(kind, kind == PH_MGS_GRID ? 0 : size);
    PH_CUDA(ctx, mgs_buffers(ctx, L, n, code));
    ctx->mgs_variant[key] = code;
  }
  // a captured path graph holds the previous choice: rebuild it on next use
  ph_track_release(ctx);
  return PH_OK;
}

namespace {
template <class P>
__global__ void k_warp_sum(const double *in, double *out) {
  typename P::real v;
#pragma unroll
  for (int l = 0; l < P::L; ++l) P::set_limb(v, l, in[threadIdx.x * P::L + l]);
  v = warp_exact_sum(v);
  if (threadIdx.x == 0)
#pragma unroll
    for (int l = 0; l < P::L; ++l) out[l] = P::limb(v, l);
}
}  // namespace

extern "C" ph_status ph_debug_warp_sum(int device, int limbs, const double *in, double *out) {
  if ((limbs != 2 && limbs != 4) || !in || !out) return PH_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return PH_ECUDA; }
  double *d = nullptr;
  const size_t nin = 32 * (size_t)limbs;
  if (cudaMalloc(&d, sizeof(double) * (nin + 4)) != cudaSuccess) { cudaGetLastError(); return PH_ENOMEM; }
  cudaError_t e = cudaMemcpy(d, in, sizeof(double) * nin, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    if (limbs == 2) k_warp_sum<DD><<<1, 32>>>(d, d + nin);
    else k_warp_sum<QD><<<1, 32>>>(d, d + nin);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d + nin, sizeof(double) * limbs, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) { cudaGetLastError(); return PH_ECUDA; }
  return PH_OK;
}

namespace {
// one case per thread: a - ar b + sg ai c in the MGS kernels' fixed-point forms
template <int L>
__global__ void k_debug_update(int count, const double *in, double *out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= count) return;
  const double *v = in + (long)c * 6 * L;
  if constexpr (L == 2) {
    const dd a = {v[0], v[1]}, ar = {v[2], v[3]}, b = {v[4], v[5]}, ai = {v[6], v[7]};
    const dd cc = {v[8], v[9]};
    const dd r = fx_upd(a, ar, b, ai, cc, v[10] < 0 ? -1.0 : 1.0);
    out[2L * c] = r.h;
    out[2L * c + 1] = r.l;
  } else {
    qd x[5];
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
      for (int l = 0; l < 4; ++l) x[q].x[l] = v[4 * q + l];
    const qd r = qf_upd(x[0], x[1], x[2], x[3], x[4], v[20] < 0 ? -1.0 : 1.0);
#pragma unroll
    for (int l = 0; l < 4; ++l) out[4L * c + l] = r.x[l];
  }
}
}  // namespace

extern "C" ph_status ph_debug_update(int device, int limbs, int count, const double *in,
                                     double *out) {
  if ((limbs != 2 && limbs != 4) || count < 1 || count > 65536 || !in || !out) return PH_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return PH_ECUDA; }
  const size_t nin = (size_t)count * 6 * limbs, nout = (size_t)count * limbs;
  double *d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * (nin + nout)) != cudaSuccess) {
    cudaGetLastError();
    return PH_ENOMEM;
  }
  cudaError_t e = cudaMemcpy(d, in, sizeof(double) * nin, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    const int grid = (count + 127) / 128;
    if (limbs == 2) k_debug_update<2><<<grid, 128>>>(count, d, d + nin);
    else k_debug_update<4><<<grid, 128>>>(count, d, d + nin);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(out, d + nin, sizeof(double) * nout, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) { cudaGetLastError(); return PH_ECUDA; }
  return PH_OK;
}
