// pathblock.cuh -- one thread block tracks one whole path (the many-path and
// serving forms).  Everything a block needs is in a Job: the homotopy (the
// target system's instruction arrays, an optional start system, gamma), the
// tracking parameters, the start point, where the end point and statistics go,
// and the job's own workspace in device memory.
//
// The step follows the same definitions as the single-path kernels (the same
// controller code, the same Newton tests, the same reverse-mode evaluation);
// the MGS inside a block is the unnormalised right-looking form with columns
// dealt round-robin to the 8 warps, the pivot norms in shared memory, and a
// block barrier per column step.
#pragma once
#include <type_traits>

#include "ctrl.h"
#include "exsum.cuh"
#include "internal.h"
#include "mp.cuh"
#include "pathdev.cuh"
#include "qfx.cuh"

namespace ph {

constexpr int kBT = 256;          // threads per block: 8 warps, 2 per SM sub-partition
constexpr int kNW = kBT / 32;
constexpr int kHistB = 16;        // accepted points kept for the predictor
constexpr int kSG = 4;            // lanes per output in the summation, until tuned

struct Job {
  int L, N, n, Mf, Mpf, maxvf, Mg, Mpg, maxvg, emax, nout;
  const int32_t *nvf, *vidxf, *vexpf, *optrf, *oslotf, *deg;
  const double *coeff_f;
  const int32_t *nvg, *vidxg, *vexpg, *optrg, *oslotg;    // null: total-degree start
  const double *coeff_g;
  const uint8_t *zrows_g;         // g's rows without terms (held fixed when p.fixed_rows)
  const double *gamma;            // [2L]
  ph_track_params p;
  const double *x0;               // [2L][n]
  double *x_out;                  // [2L][n]
  ph_path_stats *stats;           // one record (may be null)
  ph_step_record *log;            // log_cap records (may be null)
  int log_cap;
  int sum_lanes;                  // lanes per output of the summation: 1, 2, 4, ..., 32
  double *ws;                     // this job's workspace
  long o_x, o_dx, o_hist, o_ptab, o_spow, o_A, o_W, o_fslots, o_gslots, o_scal, o_t, o_g, o_h;
  long ldA, nsf, nsg;
};

// Workspace layout (doubles, 256-byte aligned regions) of a job.
struct JobLayout {
  long o_x, o_dx, o_hist, o_ptab, o_spow, o_A, o_W, o_fslots, o_gslots, o_scal, o_t, o_g, o_h, stride;
};

inline JobLayout job_layout(int L, int n, long ldA, int emax, long nsf, long nsg) {
  auto up = [](long v) { return (v + 31) / 32 * 32; };
  const long pt = 2L * L * n, nc = n + 1, ntab = emax > 2 ? emax - 1 : 1;
  JobLayout o;
  o.o_x = 0;
  o.o_dx = o.o_x + up(pt);
  o.o_hist = o.o_dx + up(pt);
  o.o_ptab = o.o_hist + up(pt * kHistB);
  o.o_spow = o.o_ptab + up(pt * ntab);
  o.o_A = o.o_spow + up(2 * pt);
  o.o_W = o.o_A + up(2L * L * nc * ldA);
  o.o_fslots = o.o_W + up(2L * L * nc * nc);
  o.o_gslots = o.o_fslots + up(2L * L * nsf);
  o.o_scal = o.o_gslots + up(2L * L * nsg);
  o.o_t = o.o_scal + up(3L * L);
  o.o_g = o.o_t + up(L);
  o.o_h = o.o_g + up(2L * L);
  o.stride = o.o_h + up(2 * ldA);
  return o;
}

// dynamic shared memory of a block for jobs of up to n variables: the back
// substitution's y [2L][n], the pivot norms [L][n+1], the columns' exponent
// bounds of the fixed-point MGS [n+1] (unsigned), and in QD the pivot column
// in fixed point [2][n] (QF)
inline size_t job_smem_bytes(int L, int n) {
  return sizeof(double) * (2L * L * n + (long)L * (n + 1) + (n + 2) / 2) +
         (L == 4 ? sizeof(QF) * 2 * (size_t)n : 0);
}

// one part (0 = real, 1 = imaginary) of element i of a complex array laid out
// [limb][re|im][...] with `plane` doubles between planes
template <class P>
PHD typename P::real rp_load(const double *v, long plane, int part, long i) {
  return r_load<P>(v + part * plane, 2 * plane, i);
}
template <class P>
PHD void rp_store(double *v, long plane, int part, long i, const typename P::real &z) {
  r_store<P>(v + part * plane, 2 * plane, i, z);
}

// the sum over the warp: exact integer sums for double-double and
// quad-double (exsum.cuh), a shuffle tree for one-limb types
template <class P>
__device__ typename P::real warp_sum_part(typename Part<P>::acc a) {
  if constexpr (std::is_same<P, DD>::value) {
    return warp_exact_sum(Part<DD>::value(a));
  } else if constexpr (std::is_same<P, QD>::value) {
    return warp_exact_sum(a.v);
  } else {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) a = Part<P>::combine(a, Part<P>::shfl(a, m));
    return Part<P>::value(a);
  }
}

// The outputs [o0, o1) of the homotopy's values and Jacobian summed by the
// block with G lanes per output (the paper's threads per sum, Section 3.3);
// put(o, value) runs on each output's first lane.
template <class P, int G, class Put>
__device__ void block_sum_g(const Job &a, int o0, int o1, const double *fslots,
                            const double *gslots, const double *spow, const double *scal,
                            Put put) {
  const int tid = threadIdx.x;
  for (int ob = o0; ob < o1; ob += kBT / G) {
    const int o = ob + tid / G, lane = tid % G;
    const bool act = o < o1;
    cx<P> val = sum_output<P, G>(act, o, lane, a.N, a.n, a.optrf, a.oslotf, fslots, a.nsf,
                                 a.optrg, a.oslotg, gslots, a.nsg, spow, scal, 1,
                                 a.p.fixed_rows ? a.zrows_g : nullptr);
    if (act && lane == 0) put(o, val);
  }
}

template <class P, class Put>
__device__ void block_sum(const Job &a, int o0, int o1, const double *fslots,
                          const double *gslots, const double *spow, const double *scal, Put put) {
  switch (a.sum_lanes) {
    case 1: block_sum_g<P, 1>(a, o0, o1, fslots, gslots, spow, scal, put); break;
    case 2: block_sum_g<P, 2>(a, o0, o1, fslots, gslots, spow, scal, put); break;
    case 8: block_sum_g<P, 8>(a, o0, o1, fslots, gslots, spow, scal, put); break;
    case 16: block_sum_g<P, 16>(a, o0, o1, fslots, gslots, spow, scal, put); break;
    case 32: block_sum_g<P, 32>(a, o0, o1, fslots, gslots, spow, scal, put); break;
    default: block_sum_g<P, 4>(a, o0, o1, fslots, gslots, spow, scal, put); break;
  }
}

// Largest exponent field of the leading limbs of column j's rows i = lane,
// lane + 32, ... (both parts), over the warp: every entry is below
// 2^(field - 1022) in magnitude.
template <class P>
__device__ __forceinline__ unsigned col_exp(const double *aj, long Ap, int N, int lane) {
  unsigned m = 0;
  for (int i = lane; i < N; i += 32)
    m = max(m, max(dbl_ef(P::lead(rp_load<P>(aj, Ap, 0, i))),
                   dbl_ef(P::lead(rp_load<P>(aj, Ap, 1, i)))));
  return __reduce_max_sync(0xffffffffu, m);
}

// MGS of [J | -h] (A) and back substitution.  Returns PH_OK or PH_NONFINITE;
// on success dx and max |dx_i| (in *s_dxmax).
//
// In double-double the dot products and updates run in fixed point
// (exsum.cuh: 16 FP64 instructions per row where the FP64 forms take 48 for a
// complex dot product, 16 for 54 for an update).  A dot product's terms are
// bounded by the product of its columns' largest entries, so each column's
// largest exponent field is kept in shared memory (s_nrm + L (n+1)) and
// refreshed when the column is updated; the accumulator's scale follows from
// the two bounds, with no pass over the rows first.  The truncation error is
// below 2^-118 of the bound per term, under 2^-107 ||a_k|| ||a_j|| in all for
// the column heights this kernel takes, below the FP64 form's.
template <class P>
__device__ int block_mgs(int N, int n, long ldA, double *A, double *W, double *dx, double *s_nrm,
                         double *s_y, double *s_dxmax) {
  typedef typename P::real real;
  typedef Part<P> PO;
  constexpr bool kDD = std::is_same<P, DD>::value;
  constexpr bool kQD = std::is_same<P, QD>::value;
  constexpr bool kFix = kDD || kQD;
  __shared__ int s_bad;
  const int nc = n + 1;
  const long Ap = (long)nc * ldA, Wp = (long)nc * nc;
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  unsigned *s_cexp = (unsigned *)(s_nrm + (long)P::L * nc);
  QF *s_piv = (QF *)(s_nrm + (long)P::L * nc + (nc + 1) / 2);   // QD: [2][N]
  const bool qcache = kQD && N <= n;               // the buffer holds n rows
  // headroom of a dot product's accumulator: 2N leading products and small terms
  const int lgN = 32 - __clz(2 * N + 1);
  if (tid == 0) s_bad = 0;
  if constexpr (kFix) {
    for (int j = w; j <= n; j += kNW) {           // a column's bound is kept by its warp
      const unsigned m = col_exp<P>(A + (long)j * ldA, Ap, N, lane);
      if (lane == 0) s_cexp[j] = m;
    }
  }
  if (w == 0) {                                    // ||a_0||^2
    typename PO::acc ar = PO::zero(), ai = PO::zero();
    for (int i = lane; i < N; i += 32) {
      PO::sq(ar, rp_load<P>(A, Ap, 0, i));
      PO::sq(ai, rp_load<P>(A, Ap, 1, i));
    }
    real s = P::add(warp_sum_part<P>(ar), warp_sum_part<P>(ai));
    if (lane == 0) r_store<P>(s_nrm, nc, 0, s);
  }
  for (int k = 0; k < n; ++k) {
    __syncthreads();
    const real r2 = r_load<P>(s_nrm, nc, k);
    const double lead = P::lead(r2);
    if (!(lead > 0.0) || !isfinite(lead)) {        // the same value in every thread
      if (tid == 0) s_bad = 1;
      break;
    }
    const real inv2 = P::recip(r2);
    const double *ak = A + (long)k * ldA;
    if constexpr (kQD) {
      if (qcache) {                                // the pivot column in fixed point, once
        for (int i = tid; i < N; i += kBT) {
          bool bad = false;
          s_piv[i] = qf_from(rp_load<P>(ak, Ap, 0, i), &bad);
          s_piv[N + i] = qf_from(rp_load<P>(ak, Ap, 1, i), &bad);
        }
        __syncthreads();
      }
    }
    for (int j = k + 1 + (((w - (k + 1)) % kNW) + kNW) % kNW; j <= n; j += kNW) {
      double *aj = A + (long)j * ldA;
      real dsr, dsi;                               // a_k^H a_j
      if constexpr (kDD) {
        const int ek = (int)s_cexp[k], ej = (int)s_cexp[j];
        const int kb = ek + ej - 1022;             // the products are below 2^(kb - 1022)
        if (ek == 0 || ej == 0) {
          dsr = dsi = DD::zero();
        } else if (ek == 0x7ff || ej == 0x7ff || kb > 2046) {
          dsr = dsi = DD::from(__longlong_as_double(0x7ff8000000000000ll));
        } else {
          const int base = fx_base(kb, lgN);
          fx128 accr = 0, acci = 0;
          for (int i = lane; i < N; i += 32) {
            const dd akr = rp_load<P>(ak, Ap, 0, i), aki = rp_load<P>(ak, Ap, 1, i);
            const dd ajr = rp_load<P>(aj, Ap, 0, i), aji = rp_load<P>(aj, Ap, 1, i);
            fx_dot2(accr, akr, ajr, aki, aji, 1.0, base);
            fx_dot2(acci, akr, aji, aki, ajr, -1.0, base);
          }
          dsr = fx_round_dd(fx_warp_sum(accr), base);
          dsi = fx_round_dd(fx_warp_sum(acci), base);
        }
      } else if constexpr (kQD) {
        const int ek = (int)s_cexp[k], ej = (int)s_cexp[j];
        const int kb = ek + ej - 1022;             // the products are below 2^(kb - 1022)
        if (ek == 0 || ej == 0) {
          dsr = dsi = QD::zero();
        } else if (ek == 0x7ff || ej == 0x7ff || kb > 2046) {
          dsr = dsi = QD::from(__longlong_as_double(0x7ff8000000000000ll));
        } else {
          // the sum of 2N products below 2^lg times the bound; three more bits
          // keep every product's shift to the accumulator non-negative
          const int lg = lgN + 3;
          const int base = kb - 1022 + lg + 1 - 255;
          Q256 accr = q_zero(), acci = q_zero();
          bool bad = false;
          for (int i = lane; i < N; i += 32) {
            const qd ajr = rp_load<P>(aj, Ap, 0, i), aji = rp_load<P>(aj, Ap, 1, i);
            if (qcache) {
              qf_dot2c(accr, s_piv[i], ajr, s_piv[N + i], aji, 1.0, base, &bad);
              qf_dot2c(acci, s_piv[i], aji, s_piv[N + i], ajr, -1.0, base, &bad);
            } else {
              const qd akr = rp_load<P>(ak, Ap, 0, i), aki = rp_load<P>(ak, Ap, 1, i);
              qf_dot2(accr, akr, ajr, aki, aji, 1.0, base, &bad);
              qf_dot2(acci, akr, aji, aki, ajr, -1.0, base, &bad);
            }
          }
#pragma unroll
          for (int m = 16; m > 0; m >>= 1) {
            accr = fix_add<4>(accr, q_shfl_xor(accr, m));
            acci = fix_add<4>(acci, q_shfl_xor(acci, m));
          }
          fix_round4(accr, base, dsr.x);
          fix_round4(acci, base, dsi.x);
          if (__any_sync(0xffffffffu, bad))
            dsr = dsi = QD::from(__longlong_as_double(0x7ff8000000000000ll));
        }
      } else {
        typename PO::acc dr = PO::zero(), di = PO::zero();
        for (int i = lane; i < N; i += 32) {
          real akr = rp_load<P>(ak, Ap, 0, i), aki = rp_load<P>(ak, Ap, 1, i);
          real ajr = rp_load<P>(aj, Ap, 0, i), aji = rp_load<P>(aj, Ap, 1, i);
          PO::dot2(dr, akr, ajr, aki, aji, 1.0);
          PO::dot2(di, akr, aji, aki, ajr, -1.0);
        }
        dsr = warp_sum_part<P>(dr);
        dsi = warp_sum_part<P>(di);
      }
      const real alr = P::mul(dsr, inv2);
      const real ali = P::mul(dsi, inv2);
      if (lane == 0) {
        rp_store<P>(W + (long)j * nc, Wp, 0, k, alr);
        rp_store<P>(W + (long)j * nc, Wp, 1, k, ali);
      }
      typename PO::acc nr = PO::zero(), ni = PO::zero();
      unsigned emax = 0;                           // the updated column's bound (DD, QD)
      QF qalr, qali;                               // alpha in fixed point (QD)
      bool abad = false;
      if constexpr (kQD) {
        qalr = qf_from(alr, &abad);
        qali = qf_from(ali, &abad);
      }
      for (int i = lane; i < N; i += 32) {
        real akr = rp_load<P>(ak, Ap, 0, i), aki = rp_load<P>(ak, Ap, 1, i);
        real ajr, aji;
        if constexpr (kDD) {
          ajr = fx_upd(rp_load<P>(aj, Ap, 0, i), alr, akr, ali, aki, 1.0);
          aji = fx_upd(rp_load<P>(aj, Ap, 1, i), alr, aki, ali, akr, -1.0);
          emax = max(emax, max(dbl_ef(ajr.h), dbl_ef(aji.h)));
        } else if constexpr (kQD) {
          if (qcache) {
            ajr = qf_upd3(rp_load<P>(aj, Ap, 0, i), qalr, s_piv[i], qali, s_piv[N + i], 1.0, abad);
            aji = qf_upd3(rp_load<P>(aj, Ap, 1, i), qalr, s_piv[N + i], qali, s_piv[i], -1.0, abad);
          } else {
            ajr = qf_upd2(rp_load<P>(aj, Ap, 0, i), qalr, akr, qali, aki, 1.0, abad);
            aji = qf_upd2(rp_load<P>(aj, Ap, 1, i), qalr, aki, qali, akr, -1.0, abad);
          }
          emax = max(emax, max(dbl_ef(ajr.x[0]), dbl_ef(aji.x[0])));
        } else {
          ajr = PO::upd(rp_load<P>(aj, Ap, 0, i), alr, akr, ali, aki, 1.0);
          aji = PO::upd(rp_load<P>(aj, Ap, 1, i), alr, aki, ali, akr, -1.0);
        }
        rp_store<P>(aj, Ap, 0, i, ajr);
        rp_store<P>(aj, Ap, 1, i, aji);
        if (j == k + 1) {
          PO::sq(nr, ajr);
          PO::sq(ni, aji);
        }
      }
      if constexpr (kFix) {
        emax = __reduce_max_sync(0xffffffffu, emax);
        if (lane == 0) s_cexp[j] = emax;
      }
      if (j == k + 1) {
        real s = P::add(warp_sum_part<P>(nr), warp_sum_part<P>(ni));
        if (lane == 0) r_store<P>(s_nrm, nc, j, s);
      }
    }
  }
  __syncthreads();
  if (s_bad) return PH_NONFINITE;
  // back substitution on y = alpha_{., n} by warp 0: dx_k = y_k, y_i -= alpha_ik dx_k
  if (w == 0) {
    const double *yc = W + (long)n * nc;
    for (int i = lane; i < n; i += 32) c_store<P>(s_y, n, i, c_load<P>(yc, Wp, i));
    __syncwarp();
    for (int k = n - 1; k >= 1; --k) {
      const real xr = rp_load<P>(s_y, n, 0, k), xi = rp_load<P>(s_y, n, 1, k);
      const double *Wk = W + (long)k * nc;
      for (int i = lane; i < k; i += 32) {
        real wr = rp_load<P>(Wk, Wp, 0, i), wi = rp_load<P>(Wk, Wp, 1, i);
        rp_store<P>(s_y, n, 0, i, PO::upd(rp_load<P>(s_y, n, 0, i), wr, xr, wi, xi, 1.0));
        rp_store<P>(s_y, n, 1, i, PO::upd(rp_load<P>(s_y, n, 1, i), wr, xi, wi, xr, -1.0));
      }
      __syncwarp();
    }
    double m = 0.0;
    for (int i = lane; i < n; i += 32) {
      cx<P> v = c_load<P>(s_y, n, i);
      c_store<P>(dx, n, i, v);
      double mg = c_mag_lead<P>(v);
      if (!(mg <= m)) m = mg;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      double o = __shfl_xor_sync(0xffffffffu, m, off);
      if (!(o <= m)) m = o;
    }
    if (lane == 0) *s_dxmax = m;
  }
  __syncthreads();
  return PH_OK;
}

// The Newton system of the mixed-precision corrector, solved in precision LP
// (F64 or F32) by the calling block: the Jacobian at x rounded to LP (power
// table, reverse-mode terms and summation in LP, written to the workspace's
// regions in the one-limb layout), the right-hand side -h (hl: its leading
// limbs, [re|im][ldA]) scaled by 2^-e and rounded to LP, then MGS and back
// substitution in LP.  On return dx holds d ([re|im][n], widened to double)
// with J d = -2^-e h, *s_dxmax = max |d_i| and *s_kappa = max r_kk / min r_kk
// (infinite if the factorization failed).  Returns PH_OK or PH_NONFINITE.
template <class P, class LP>
__device__ int lowprec_solve(const Job &a, const double *x, const double *tl, const double *hl,
                             int e, double *ptab, double *spow, double *scal, double *fslots,
                             double *gslots, double *A, double *W, double *dx, double *s_nrm,
                             double *s_y, double *s_dxmax, double *s_kappa) {
  const int n = a.n, N = a.N, tid = threadIdx.x, nN = n * N;
  const bool total_degree = a.optrg == nullptr;
  const long Ap = (long)(n + 1) * a.ldA;
  __syncthreads();                                 // the working-precision tables are done
  for (int j = tid; j < n; j += kBT)
    prep_variable<LP>(j, x, n, a.emax, ptab, a.deg, total_degree ? spow : nullptr);
  if (tid == 0) prep_factors<LP>(tl, a.gamma, a.p.relax_k, scal);
  for (int i = tid; i < N; i += kBT)
    c_store<LP>(A + (long)n * a.ldA, Ap, i,
                c_from<LP>(ldexp(hl[i], -e), ldexp(hl[a.ldA + i], -e)));
  __syncthreads();
  for (int s = tid; s < a.Mf; s += kBT)
    ad_term<LP>(s, a.Mpf, a.nvf, a.vidxf, a.vexpf, a.coeff_f, ptab, n, a.maxvf, fslots, a.nsf);
  for (int s = tid; s < a.Mg; s += kBT)
    ad_term<LP>(s, a.Mpg, a.nvg, a.vidxg, a.vexpg, a.coeff_g, ptab, n, a.maxvg, gslots, a.nsg);
  __syncthreads();
  block_sum<LP>(a, 0, nN, fslots, gslots, spow, scal, [&](int o, const cx<LP> &val) {
    const int j = o / N, i = o - j * N;
    c_store<LP>(A + (long)j * a.ldA, Ap, i, val);
  });
  __syncthreads();
  const int ms = block_mgs<LP>(N, n, a.ldA, A, W, dx, s_nrm, s_y, s_dxmax);
  if (tid == 0) {
    double mx = 0.0, mn = INFINITY;
    for (int k = 0; k < n; ++k) {
      const double v = LP::lead(r_load<LP>(s_nrm, n + 1, k));
      mx = fmax(mx, v);
      mn = fmin(mn, v);
    }
    *s_kappa = ms == PH_OK ? sqrt(mx / mn) : INFINITY;
  }
  __syncthreads();
  return ms;
}

// Tracks the job's path from its start point to its end with the calling
// block (kBT threads); writes the end point (the last accepted point), the
// statistics and the step log.  smem: dynamic shared memory for n variables.
template <class P>
__device__ void track_job(const Job &a, double *smem) {
  typedef typename P::real real;
  double *s_y = smem;                                   // [2L][n]
  double *s_nrm = smem + 2 * P::L * a.n;                // [L][n+1]
  __shared__ ph_ctrl_state s_ctrl;
  __shared__ real s_w[kHistB];
  __shared__ double s_t[kHistB];
  __shared__ int s_head, s_count, s_dec, s_ok, s_upd, s_iters, s_bad;
  __shared__ double s_tn, s_last, s_res, s_dxn, s_dxmax, s_xmax;
  __shared__ unsigned long long s_resbits;
  __shared__ ph_path_stats s_st;
  __shared__ int s_lin, s_scale_e, s_force, s_escalate, s_onpath, s_linear, s_wp;
  __shared__ double s_dxn2;
  __shared__ double s_cond, s_kappa;

  const int n = a.n, N = a.N, tid = threadIdx.x;
  const long pt = 2L * P::L * n;
  double *ws = a.ws;
  double *x = ws + a.o_x, *dx = ws + a.o_dx, *hist = ws + a.o_hist, *ptab = ws + a.o_ptab;
  double *spow = ws + a.o_spow, *A = ws + a.o_A, *W = ws + a.o_W, *fslots = ws + a.o_fslots;
  double *gslots = ws + a.o_gslots, *scal = ws + a.o_scal, *tl = ws + a.o_t;
  const bool fixed = a.p.fixed_steps > 0;
  const long Ap = (long)(n + 1) * a.ldA;
  const bool total_degree = a.optrg == nullptr;
  double *hl = ws + a.o_h;                              // leading limbs of -h: [re|im][ldA]
  const double endgame = a.p.endgame_t > 0.0 ? a.p.endgame_t : 1.0;
  const double cond32 = a.p.cond_f32 > 0.0 ? a.p.cond_f32 : 1e3;

  // start: the start point is the only accepted point
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (long e = tid; e < pt; e += kBT) {
    double v = a.x0[e];
    hist[e] = v;
    if (!isfinite(v)) s_bad = 1;
  }
  if (tid == 0) {
    ctrl_init(&s_ctrl, &a.p);
    memset(&s_st, 0, sizeof s_st);
    s_cond = INFINITY;
    s_wp = 0;
    s_head = 0;
    s_count = 1;
    s_t[0] = 0.0;
  }
  __syncthreads();
  if (s_bad) {
    for (long e = tid; e < pt; e += kBT) a.x_out[e] = a.x0[e];
    if (tid == 0 && a.stats) {
      s_st.status = PH_NONFINITE;
      *a.stats = s_st;
    }
    __syncthreads();
    return;
  }
  for (;;) {
    if (tid == 0) s_tn = ctrl_next_t(&s_ctrl, &a.p);
    __syncthreads();
    const double tn = s_tn;
    if (tn < 0.0) break;
    // predictor: Lagrange weights of the last m accepted points at tn
    const int m = s_count < a.p.pred_order + 1 ? s_count : a.p.pred_order + 1;
    if (tid < m) {
      const int sj = (s_head - (m - 1 - tid) + kHistB) % kHistB;
      const double tj = s_t[sj];
      real num = P::from(1.0), den = P::from(1.0);
      for (int l = 0; l < m; ++l) {
        if (l == tid) continue;
        const double tq = s_t[(s_head - (m - 1 - l) + kHistB) % kHistB];
        double s1, e1;
        real u = P::zero(), v = P::zero();
        two_sum(tn, -tq, s1, e1);
        P::set_limb(u, 0, s1);
        if (P::L > 1) P::set_limb(u, 1, e1);
        two_sum(tj, -tq, s1, e1);
        P::set_limb(v, 0, s1);
        if (P::L > 1) P::set_limb(v, 1, e1);
        num = P::mul(num, u);
        den = P::mul(den, v);
      }
      s_w[tid] = m == 1 ? P::from(1.0) : P::div(num, den);
    }
    if (tid == 0) {
      tl[0] = tn;
      for (int l = 1; l < P::L; ++l) tl[l] = 0.0;
      s_force = 0;
    }
    // A step whose mixed-precision corrector fails is corrected once more from
    // the predicted point one precision up (pass 1) before it counts as failed,
    // wherever the working-precision corrector might have decided otherwise:
    // in double if it solved in single by request (lin_prec 2); in working
    // precision if a double solve had kappa u_double above kEscalateRho (the
    // estimate is only a lower bound of kappa) or if it failed although an
    // update below sqrt(tol_dx) was followed by another one (the working-
    // precision corrector would have succeeded there), or if its last three
    // updates contracted more slowly than quadratically (linear_contraction:
    // its solves limit it, whatever the estimate shows; the rest of the path
    // then runs in working precision).  A corrector that fails while its
    // updates are still large takes the working-precision iterates, to
    // kappa u_low, and fails as that one would: the step size halves.
    for (int pass = 0;; ++pass) {
      if (tid == 0) {
        s_last = a.p.max_res;
        s_dec = 0;
        s_ok = fixed ? 1 : 0;
        s_upd = 0;
        s_iters = 0;
        s_escalate = 0;
        s_onpath = 0;
        s_linear = 0;
      }
      __syncthreads();
      for (int i = tid; i < n; i += kBT) {
        cx<P> acc = c_zero<P>();
        for (int j = 0; j < m; ++j) {
          const int sj = (s_head - (m - 1 - j) + kHistB) % kHistB;
          acc = c_add<P>(acc, c_mul_real<P>(c_load<P>(hist + sj * pt, n, i), s_w[j]));
        }
        c_store<P>(x, n, i, acc);
      }
      // corrector (Fig. 2)
      // One iteration beyond max_newton for a low-precision corrector whose
      // previous update was below sqrt(tol_dx): the working-precision corrector
      // would have squared that update below tol_dx and succeeded by now, while
      // the low-precision one contracts only by kappa u_low per iteration.
      const int max_it = fixed ? a.p.max_newton : a.p.max_newton + 1;
      for (int it = 0; it < max_it; ++it) {
        __syncthreads();
        if (tid == 0) {                              // the precision of this iteration's solve
          int lin = a.p.lin_prec;
          if (tn >= endgame || s_force == 2 || s_wp) lin = 0;
          // automatic: single on a step's first iteration and while the current
          // error, estimated as the square of the last update, is at least the
          // single-precision solve's relative error kappa u_single
          if (lin == 3)
            lin = s_cond <= cond32 && (it == 0 || s_dxn * s_dxn >= s_cond * 0x1p-24) ? 2 : 1;
          if (s_force == 1 && lin == 2) lin = 1;
          s_lin = lin;
          s_resbits = 0ull;
        }
        for (int j = tid; j < n; j += kBT)
          prep_variable<P>(j, x, n, a.emax, ptab, a.deg, total_degree ? spow : nullptr);
        if (tid == 0) prep_factors<P>(tl, a.gamma, a.p.relax_k, scal);
        __syncthreads();
        const int lin = s_lin;
        double mymax = 0.0;
        if (lin == 0) {
          // h and J in working precision into A = [J | -h]
          for (int s = tid; s < a.Mf; s += kBT)
            ad_term<P>(s, a.Mpf, a.nvf, a.vidxf, a.vexpf, a.coeff_f, ptab, n, a.maxvf, fslots, a.nsf);
          for (int s = tid; s < a.Mg; s += kBT)
            ad_term<P>(s, a.Mpg, a.nvg, a.vidxg, a.vexpg, a.coeff_g, ptab, n, a.maxvg, gslots, a.nsg);
          __syncthreads();
          block_sum<P>(a, 0, a.nout, fslots, gslots, spow, scal, [&](int o, const cx<P> &val) {
            if (o < n * N) {
              const int j = o / N, i = o - j * N;
              c_store<P>(A + (long)j * a.ldA, Ap, i, val);
            } else {
              const int i = o - n * N;
              c_store<P>(A + (long)n * a.ldA, Ap, i, c_neg<P>(val));
              double mg = c_mag_lead<P>(val);
              if (!(mg <= mymax)) mymax = mg;
            }
          });
        } else {
          // the residual alone in working precision; the leading limbs of -h to hl
          for (int s = tid; s < a.Mf; s += kBT)
            val_term<P>(s, a.Mpf, a.nvf, a.vidxf, a.vexpf, a.coeff_f, ptab, n, a.emax, a.maxvf,
                        fslots, a.nsf);
          for (int s = tid; s < a.Mg; s += kBT)
            val_term<P>(s, a.Mpg, a.nvg, a.vidxg, a.vexpg, a.coeff_g, ptab, n, a.emax, a.maxvg,
                        gslots, a.nsg);
          __syncthreads();
          block_sum<P>(a, n * N, n * N + N, fslots, gslots, spow, scal,
                       [&](int o, const cx<P> &val) {
            const int i = o - n * N;
            hl[i] = -P::lead(val.re);
            hl[a.ldA + i] = -P::lead(val.im);
            double mg = c_mag_lead<P>(val);
            if (!(mg <= mymax)) mymax = mg;
          });
        }
        atomicMax(&s_resbits, (unsigned long long)__double_as_longlong(mymax));
        __syncthreads();
        if (tid == 0) {                              // residual test
          const double r = __longlong_as_double((long long)s_resbits);
          s_res = r;
          s_iters += 1;
          s_st.newton_iters += 1;
          s_st.res = r;
          if (!fixed) {
            if (!(r <= s_last) || !isfinite(r)) { s_dec = 1; s_ok = 0; }
            else if (r < ctrl_tol_res(&a.p, s_tn)) { s_dec = 1; s_ok = 1; }
          }
          s_scale_e = (r > 0.0 && isfinite(r)) ? ilogb(r) : 0;
        }
        __syncthreads();
        if (s_dec) break;
        int ms;
        if (lin == 0) {
          ms = block_mgs<P>(N, n, a.ldA, A, W, dx, s_nrm, s_y, &s_dxmax);
        } else {
          ms = lin == 2 ? lowprec_solve<P, F32>(a, x, tl, hl, s_scale_e, ptab, spow, scal, fslots,
                                                gslots, A, W, dx, s_nrm, s_y, &s_dxmax, &s_kappa)
                        : PH_NONFINITE;
          double u_lin = 0x1p-24;                    // unit roundoff of the solve used
          if (lin == 2 && tid == 0) {
            if (ms == PH_OK) s_st.solves_f32 += 1;
            s_cond = ms == PH_OK ? s_kappa : INFINITY;
          }
          if (lin == 1 || ms != PH_OK) {             // double (also the retry of a failed single)
            ms = lowprec_solve<P, F64>(a, x, tl, hl, s_scale_e, ptab, spow, scal, fslots, gslots, A,
                                       W, dx, s_nrm, s_y, &s_dxmax, &s_kappa);
            u_lin = 0x1p-53;
            if (tid == 0) {
              s_st.solves_f64 += 1;
              s_cond = ms == PH_OK ? s_kappa : INFINITY;
            }
          }
          if (tid == 0) {
            s_st.cond = s_cond;
            if (u_lin > 0x1p-53) {
              if (a.p.lin_prec == 2) s_escalate = max(s_escalate, 1);  // single by request
            } else if (!(s_cond * u_lin <= kEscalateRho)) {
              s_escalate = 2;
            }
          }
        }
        if (ms != PH_OK && !fixed) {
          if (tid == 0) { s_dec = 1; s_ok = 0; }
          __syncthreads();
          break;
        }
        const int e = s_scale_e;
        for (int i = tid; i < n; i += kBT) {
          cx<P> d;
          if (ms != PH_OK) {
            d = c_from<P>(NAN, NAN);
          } else if (lin == 0) {
            d = c_load<P>(dx, n, i);
          } else {
            d = c_from<P>(ldexp(dx[i], e), ldexp(dx[n + i], e));
          }
          c_store<P>(x, n, i, c_add<P>(c_load<P>(x, n, i), d));
        }
        if (tid == 0) {                              // update test
          const double d = ms != PH_OK ? NAN : (lin == 0 ? s_dxmax : ldexp(s_dxmax, e));
          const double tol_dx = ctrl_tol_dx(&a.p, s_tn);
          const bool prev_on_path = lin != 0 && s_upd >= 1 && s_dxn <= sqrt(tol_dx);
          if (prev_on_path) s_onpath = 1;
          if (lin != 0 && s_upd >= 2 && linear_contraction(s_dxn2, s_dxn, d)) s_linear = 1;
          s_dxn2 = s_dxn;
          s_dxn = d;
          s_st.dx = d;
          s_upd += 1;
          s_st.updates += 1;
          if (!fixed) {
            if (!isfinite(d)) { s_dec = 1; s_ok = 0; }
            else if (d < tol_dx) { s_dec = 1; s_ok = 1; }
            else s_last = s_res;
          }
          if (!s_dec && s_iters >= a.p.max_newton && !(prev_on_path && s_iters < max_it)) {
            s_dec = 1;
            s_ok = fixed ? 1 : 0;
          }
        }
        __syncthreads();
        if (s_dec) break;
      }
      __syncthreads();
      // a low-precision corrector that failed after an update below
      // sqrt(tol_dx) followed by another: the working-precision corrector
      // would have succeeded
      if (tid == 0 && !s_ok && s_onpath) s_escalate = 2;
      // a low-precision corrector that failed while contracting only linearly:
      // its solves limit it, the working-precision corrector might not fail;
      // the rest of the path runs in working precision
      if (tid == 0 && !s_ok && s_linear && !fixed) {
        s_escalate = 2;
        s_wp = 1;
        s_st.wp_rest = 1;
      }
      __syncthreads();
      if (pass == 0 && !s_ok && s_escalate && !fixed) {
        if (tid == 0) {
          s_force = s_escalate;
          s_st.escalated += 1;
        }
        __syncthreads();
        continue;
      }
      break;
    }
    // step control (Fig. 3)
    if (tid == 0) {
      const int ok = s_ok;
      s_st.steps += 1;
      if (ok) s_st.accepted += 1; else s_st.rejected += 1;
      if (a.log && s_st.steps <= a.log_cap) {
        ph_step_record r;
        r.t = tn;
        r.res = s_res;
        r.dx = s_dxn;
        r.accepted = ok;
        r.updates = s_upd;
        a.log[s_st.steps - 1] = r;
      }
      ctrl_report(&s_ctrl, &a.p, tn, ok);
      if (ok) {
        s_head = (s_head + 1) % kHistB;
        s_t[s_head] = tn;
        s_count = s_count < kHistB ? s_count + 1 : kHistB;
      }
      s_xmax = 0.0;
    }
    __syncthreads();
    if (s_ok) {
      double mymax = 0.0;
      for (int i = tid; i < n; i += kBT) {
        cx<P> xi = c_load<P>(x, n, i);
        c_store<P>(hist + s_head * pt, n, i, xi);
        double mg = c_mag_lead<P>(xi);
        if (!(mg <= mymax)) mymax = mg;
      }
      atomicMax((unsigned long long *)&s_xmax, (unsigned long long)__double_as_longlong(mymax));
      __syncthreads();
      if (tid == 0 && !fixed && !s_ctrl.done && !(s_xmax <= a.p.max_x)) {
        s_ctrl.done = 1;
        s_ctrl.status = PH_DIVERGED;
      }
    }
    __syncthreads();
    if (s_ctrl.done) break;
  }
  // end point: the last accepted point
  for (long e = tid; e < pt; e += kBT) a.x_out[e] = hist[(long)s_head * pt + e];
  if (tid == 0 && a.stats) {
    s_st.status = s_ctrl.status;
    s_st.t_final = s_t[s_head];
    s_st.launches = 0;
    *a.stats = s_st;
  }
  __syncthreads();
}

}  // namespace ph
