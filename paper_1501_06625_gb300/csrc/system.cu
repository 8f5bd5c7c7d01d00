// system.cu -- ph_system_load / ph_system_free: validation of a fully expanded
// polynomial system and its packing into the device layout the evaluation
// kernels read (Section 3.2):
//  - terms sorted by their number of variables v, largest first (stable), so
//    the threads of a warp run products of the same length;
//  - variable indices and exponents stored position-major, [position][term],
//    so that at each position consecutive threads read consecutive words;
//  - the reverse-mode results of term s at position p (the partial derivative
//    with respect to its p-th variable) go to slot p*Mp + s, its value to slot
//    maxv*Mp + s;
//  - for every output (Jacobian entry (i,j) at j*N + i, then value i at n*N + i)
//    the list of slots to add, in the order of the terms of polynomial i.
// Everything crosses to the device once, at load time (Section 3.1).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>

#include "internal.h"

// threads per monomial of v variables: enough that each lane's chunk has
// about four positions (the reverse sweep dominates), at most 8
int ph_ad_lanes(int v) {
  if (v <= 5) return 1;
  if (v <= 10) return 2;
  if (v <= 24) return 4;
  return 8;
}

static ph_status upload(ph_system *s, DevBuf &b, const void *src, size_t bytes) {
  cudaError_t e = b.ensure(bytes);
  if (e != cudaSuccess) return ph_cuda_fail(s->ctx, e, "cudaMalloc (system)");
  if (bytes) {
    e = cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, s->ctx->stream);
    if (e != cudaSuccess) return ph_cuda_fail(s->ctx, e, "cudaMemcpyAsync (system)");
  }
  return PH_OK;
}

extern "C" ph_status ph_system_load(ph_ctx *ctx, ph_prec prec, int N, int n,
                                    const int32_t *term_ptr, const int32_t *var_ptr,
                                    const int32_t *var_idx, const int32_t *var_exp,
                                    const double *coeff, ph_system **out) {
  if (!ctx) return PH_EINVAL;
  if (!out) return ph_fail(ctx, PH_EINVAL, "ph_system_load: out is NULL");
  *out = nullptr;
  if (prec != PH_D && prec != PH_DD && prec != PH_QD)
    return ph_fail(ctx, PH_EINVAL, "ph_system_load: prec must be PH_D, PH_DD or PH_QD");
  if (n < 1 || N < n) return ph_fail(ctx, PH_EINVAL, "ph_system_load: need N >= n >= 1");
  if ((long)n * N > (1L << 30)) return ph_fail(ctx, PH_EINVAL, "ph_system_load: system too large");
  if (!term_ptr || !var_ptr) return ph_fail(ctx, PH_EINVAL, "ph_system_load: NULL pointer array");
  const int L = (int)prec;
  if (term_ptr[0] != 0) return ph_fail(ctx, PH_EINVAL, "ph_system_load: term_ptr[0] != 0");
  for (int i = 0; i < N; ++i)
    if (term_ptr[i + 1] < term_ptr[i]) return ph_fail(ctx, PH_EINVAL, "ph_system_load: term_ptr decreases");
  const int M = term_ptr[N];
  if (M > 0 && !coeff) return ph_fail(ctx, PH_EINVAL, "ph_system_load: coeff is NULL");
  if (var_ptr[0] != 0) return ph_fail(ctx, PH_EINVAL, "ph_system_load: var_ptr[0] != 0");
  int maxv = 0, emax = 1;
  for (int k = 0; k < M; ++k) {
    if (var_ptr[k + 1] < var_ptr[k]) return ph_fail(ctx, PH_EINVAL, "ph_system_load: var_ptr decreases");
    maxv = std::max(maxv, var_ptr[k + 1] - var_ptr[k]);
  }
  const int nnz = var_ptr[M];
  if (nnz > 0 && (!var_idx || !var_exp)) return ph_fail(ctx, PH_EINVAL, "ph_system_load: NULL var arrays");
  for (int p = 0; p < nnz; ++p) {
    if (var_idx[p] < 0 || var_idx[p] >= n) return ph_fail(ctx, PH_EINVAL, "ph_system_load: variable index out of range");
    if (var_exp[p] < 1 || var_exp[p] > 4096) return ph_fail(ctx, PH_EINVAL, "ph_system_load: exponent must be in [1, 4096]");
    emax = std::max(emax, var_exp[p]);
  }
  {
    std::vector<int> seen(n, -1);
    for (int k = 0; k < M; ++k)
      for (int p = var_ptr[k]; p < var_ptr[k + 1]; ++p) {
        if (seen[var_idx[p]] == k) return ph_fail(ctx, PH_EINVAL, "ph_system_load: repeated variable in a term");
        seen[var_idx[p]] = k;
      }
  }
  if (emax > 64) return ph_fail(ctx, PH_EINVAL, "ph_system_load: exponents above 64 are not supported");

  static std::atomic<uint64_t> next_serial{1};
  ph_system *s = new (std::nothrow) ph_system();
  if (!s) return ph_fail(ctx, PH_ENOMEM, "ph_system_load: out of host memory");
  s->ctx = ctx;
  s->serial = next_serial.fetch_add(1);
  s->L = L; s->N = N; s->n = n; s->M = M; s->maxv = maxv; s->emax = emax;
  s->Mp = std::max(32, (M + 31) / 32 * 32);
  const int Mp = s->Mp;

  // degrees (total-degree start system)
  s->h_deg.assign(N, 0);
  std::vector<int> term_poly(M);
  for (int i = 0; i < N; ++i)
    for (int k = term_ptr[i]; k < term_ptr[i + 1]; ++k) {
      term_poly[k] = i;
      int d = 0;
      for (int p = var_ptr[k]; p < var_ptr[k + 1]; ++p) d += var_exp[p];
      s->h_deg[i] = std::max(s->h_deg[i], d);
    }
  s->max_deg = N ? *std::max_element(s->h_deg.begin(), s->h_deg.end()) : 0;

  // sort terms by number of variables, largest first (stable)
  std::vector<int> perm(M), inv(M);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) {
    return (var_ptr[a + 1] - var_ptr[a]) > (var_ptr[b + 1] - var_ptr[b]);
  });
  for (int sidx = 0; sidx < M; ++sidx) inv[perm[sidx]] = sidx;

  std::vector<int32_t> poly(Mp, -1), nv(Mp, 0);
  std::vector<int32_t> vidx((size_t)std::max(maxv, 1) * Mp, 0), vexp((size_t)std::max(maxv, 1) * Mp, 1);
  std::vector<double> co((size_t)2 * L * Mp, 0.0);
  for (int sidx = 0; sidx < M; ++sidx) {
    int k = perm[sidx];
    poly[sidx] = term_poly[k];
    nv[sidx] = var_ptr[k + 1] - var_ptr[k];
    for (int p = 0; p < nv[sidx]; ++p) {
      vidx[(size_t)p * Mp + sidx] = var_idx[var_ptr[k] + p];
      vexp[(size_t)p * Mp + sidx] = var_exp[var_ptr[k] + p];
    }
    for (int c = 0; c < 2 * L; ++c) co[(size_t)c * Mp + sidx] = coeff[(size_t)c * M + k];
  }

  // lanes per monomial by its number of variables (terms are sorted, so each
  // lane count covers a contiguous range)
  for (int sidx = 0; sidx < M;) {
    int lanes = ph_ad_lanes(nv[sidx]);
    int e = sidx;
    while (e < M && ph_ad_lanes(nv[e]) == lanes) ++e;
    s->buckets.push_back({sidx, e, lanes});
    sidx = e;
  }

  // summation lists
  const long nJ = (long)n * N;
  s->nout = (int)(nJ + N);
  std::vector<int32_t> optr(s->nout + 1, 0);
  for (int k = 0; k < M; ++k) {
    int i = term_poly[k];
    optr[nJ + i + 1]++;
    for (int p = var_ptr[k]; p < var_ptr[k + 1]; ++p) optr[(long)var_idx[p] * N + i + 1]++;
  }
  for (int o = 0; o < s->nout; ++o) {
    s->max_contrib = std::max(s->max_contrib, optr[o + 1]);
    optr[o + 1] += optr[o];
  }
  std::vector<int32_t> oslot(std::max(1, optr[s->nout])), fill(optr.begin(), optr.end() - 1);
  for (int k = 0; k < M; ++k) {          // terms in their given order
    int i = term_poly[k], sidx = inv[k];
    oslot[fill[nJ + i]++] = maxv * Mp + sidx;
    for (int p = var_ptr[k]; p < var_ptr[k + 1]; ++p)
      oslot[fill[(long)var_idx[p] * N + i]++] = (p - var_ptr[k]) * Mp + sidx;
  }
  if ((long)(maxv + 1) * Mp > (1L << 31) / 2) {
    delete s;
    return ph_fail(ctx, PH_EINVAL, "ph_system_load: too many terms");
  }

  std::vector<int32_t> degv(s->h_deg.begin(), s->h_deg.end());
  std::vector<uint8_t> zrows(N);
  for (int i = 0; i < N; ++i) zrows[i] = term_ptr[i + 1] == term_ptr[i] ? 1 : 0;
  ph_status st;
  if ((st = upload(s, s->poly, poly.data(), sizeof(int32_t) * Mp)) != PH_OK ||
      (st = upload(s, s->nv, nv.data(), sizeof(int32_t) * Mp)) != PH_OK ||
      (st = upload(s, s->vidx, vidx.data(), sizeof(int32_t) * vidx.size())) != PH_OK ||
      (st = upload(s, s->vexp, vexp.data(), sizeof(int32_t) * vexp.size())) != PH_OK ||
      (st = upload(s, s->coeff, co.data(), sizeof(double) * co.size())) != PH_OK ||
      (st = upload(s, s->deg, degv.data(), sizeof(int32_t) * N)) != PH_OK ||
      (st = upload(s, s->out_ptr, optr.data(), sizeof(int32_t) * optr.size())) != PH_OK ||
      (st = upload(s, s->out_slot, oslot.data(), sizeof(int32_t) * oslot.size())) != PH_OK ||
      (st = upload(s, s->zero_rows, zrows.data(), (size_t)N)) != PH_OK) {
    ph_system_free(s);
    return st;
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) {
    ph_system_free(s);
    return ph_cuda_fail(ctx, e, "cudaStreamSynchronize (system load)");
  }
  *out = s;
  return PH_OK;
}

extern "C" ph_status ph_system_free(ph_system *s) {
  if (!s) return PH_EINVAL;
  s->poly.release(); s->nv.release(); s->vidx.release(); s->vexp.release();
  s->coeff.release(); s->deg.release(); s->out_ptr.release(); s->out_slot.release();
  s->zero_rows.release();
  delete s;
  return PH_OK;
}
