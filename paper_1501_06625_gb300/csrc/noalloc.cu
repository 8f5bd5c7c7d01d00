// noalloc.cu -- ph_mgs_solve_static: a least-squares solve like
// ph_mgs_solve for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: processes whose device memory is fully
// reserved by another allocator (a framework's caching allocator, a fixed
// arena), so that a further allocation would fail or evict the owner's
// buffers, and real-time loops where an allocation's implicit device
// synchronisation is not acceptable.  This entry point allocates nothing.
// Its scratch memory (the augmented matrix, the projections, the pivot norms
// and flags, the solution, the status words) is one file-scope device array
// of kScratchBytes, which every GPU that loads the library holds until the
// process exits.
//
// The host cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the first call on each device looks the
// address up with cudaGetSymbolAddress, with that device current, and keeps
// it.  All calls share the one array: calls that overlap on the GPU (other
// streams, other host threads) race and must be serialised by the caller.
// What must start at zero (the status words and the pivot flags) is cleared
// on the caller's stream at the start of every call.
//
// The solve always runs the grid MGS kernel (one block per column); it does
// not time the cluster variant the way a context does.  Its results agree
// with ph_mgs_solve to the solver's rounding tolerance, not bit for bit.
// The call ends by reading the status and residual back to the host and
// synchronising its stream, so a stream that is being captured into a graph
// is refused with PH_EINVAL before anything is enqueued on it.
#include <mutex>

#include "internal.h"

namespace {

constexpr size_t kScratchBytes = 4u << 20;     // 4 MiB
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_addr[kMaxDevices] = {};
int g_sms[kMaxDevices] = {};

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

cudaError_t ph_mgs_launch_buffers(int sm_count, cudaStream_t stream, int L, int N, int n,
                                  double *A, long ldA, double *W, double *nrm2, double *dx,
                                  int *ready, PathState *st, double *resid);
long ph_lda(int N);

extern "C" ph_status ph_mgs_solve_static(int device, void *cuda_stream, ph_prec prec, int N,
                                         int n, const double *J, const double *rhs, double *dx,
                                         double *resid_norm) {
  if (prec != PH_D && prec != PH_DD && prec != PH_QD) return PH_EINVAL;
  if (n < 1 || N < n || !J || !rhs || !dx) return PH_EINVAL;
  if (device < 0 || device >= kMaxDevices) return PH_EINVAL;
  const int L = (int)prec, nc = n + 1;
  const long ldA = ph_lda(N), Ap = (long)nc * ldA;
  // layout of the scratch array: state | A | W | norms | pivot flags | dx | residual
  const size_t o_st = 0;
  const size_t o_A = o_st + align256(sizeof(PathState));
  const size_t o_W = o_A + align256(sizeof(double) * 2 * L * (size_t)Ap);
  const size_t o_n = o_W + align256(sizeof(double) * 2 * L * (size_t)nc * nc);
  const size_t o_i = o_n + align256(sizeof(double) * 2 * L * (size_t)nc);
  const size_t o_x = o_i + align256(sizeof(int) * (size_t)nc);
  const size_t o_r = o_x + align256(sizeof(double) * 2 * L * (size_t)n);
  const size_t need = o_r + align256(sizeof(double));
  if (need > kScratchBytes) return PH_EINVAL;    // too large for the static scratch

  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) { cudaGetLastError(); return PH_ECUDA; }
  if (prev != device && cudaSetDevice(device) != cudaSuccess) { cudaGetLastError(); return PH_ECUDA; }
  ph_status status = PH_OK;
  unsigned char *base = nullptr;
  int sms = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        status = PH_ECUDA;
      } else if (cudaDeviceGetAttribute(&g_sms[device], cudaDevAttrMultiProcessorCount, device) !=
                 cudaSuccess) {
        cudaGetLastError();
        status = PH_ECUDA;
      } else {
        g_addr[device] = (unsigned char *)p;
      }
    }
    base = g_addr[device];
    sms = g_sms[device];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (status == PH_OK) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
      cudaGetLastError();
      status = PH_ECUDA;
    } else if (cs != cudaStreamCaptureStatusNone) {
      status = PH_EINVAL;                        // nothing was enqueued on the stream
    }
  }
  PathState *st = (PathState *)(base + o_st);
  double *A = (double *)(base + o_A), *W = (double *)(base + o_W), *nrm2 = (double *)(base + o_n);
  int *ready = (int *)(base + o_i);
  double *xo = (double *)(base + o_x), *res = (double *)(base + o_r);
  PathState hs;
  double rn = 0.0;
  cudaError_t e = cudaSuccess;
  if (status == PH_OK) {
    e = cudaMemsetAsync(st, 0, sizeof(PathState), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ready, 0, sizeof(int) * (size_t)nc, s);
    for (int c = 0; c < 2 * L && e == cudaSuccess; ++c)
      e = cudaMemcpy2DAsync(A + c * Ap, ldA * sizeof(double), J + (long)c * n * N, N * sizeof(double),
                            N * sizeof(double), n, cudaMemcpyDefault, s);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(A + (long)n * ldA, Ap * sizeof(double), rhs, N * sizeof(double),
                            N * sizeof(double), 2 * L, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = ph_mgs_launch_buffers(sms, s, L, N, n, A, ldA, W, nrm2, xo, ready, st, res);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dx, xo, sizeof(double) * 2 * L * n, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&rn, res, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hs, st, sizeof hs, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      status = PH_ECUDA;
    } else if (hs.timeout) {
      status = PH_TIMEOUT;
    } else if (hs.mgs_status != PH_OK) {
      status = (ph_status)hs.mgs_status;
    } else if (resid_norm) {
      *resid_norm = rn;
    }
  }
  if (prev != device) cudaSetDevice(prev);
  return status;
}
