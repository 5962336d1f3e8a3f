// tmg_coarse_solve_noalloc: the coarse solve of the cycle for callers that cannot allocate device
// memory -- code running while a CUDA stream is being captured into a graph, memory-pool-managed
// or embedded hosts that forbid cudaMalloc/cudaFree on their call paths, and real-time loops
// where an allocation's implicit synchronisation is not acceptable.
//
// The call takes the caller's device vectors and the context's coarse operator (built earlier by
// tmg_setup) and runs the same persistent GMRES kernel as tmg_coarse_solve, but all of its
// scratch (Krylov basis, partial sums, Hessenberg, counters) lives in one file-scope device array
// of TMG_NOALLOC_SCRATCH_BYTES.  That array exists on every GPU that loads the library, until the
// process exits.  Host code only knows the array by a host-side stand-in symbol, so its device
// address is looked up once per device with cudaGetSymbolAddress (with that device current) and
// cached; that lookup happens in the first call on each device, which should therefore come before
// any stream capture.  All calls share the array: two calls that overlap on the GPU (different
// streams, or different contexts on one device) race on it.
#include <exception>
#include <mutex>
#include <new>
#include <string>

#include "tmg_host.h"

#define TMG_NOALLOC_SCRATCH_BYTES ((size_t)32 << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[TMG_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_lock;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on `device` (which must be current).
int scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return TMG_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_lock);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return TMG_ERR_CUDA;
    g_scratch_addr[device] = p;
  }
  *out = g_scratch_addr[device];
  return TMG_OK;
}

template <typename A2, typename B2>
__global__ void k_noalloc_convert(const A2* __restrict__ a, B2* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const A2 v = a[i];
    B2 o;
    o.x = v.x;
    o.y = v.y;
    b[i] = o;
  }
}

}  // namespace

extern "C" int tmg_coarse_solve_noalloc(tmg_ctx* ctx, const double* b, double* x, double mu, int prec) {
  if (!ctx) return TMG_ERR_ARG;
  tmg::Ctx& c = ctx->c;
  try {
    if (!b || !x || (prec != TMG_PREC_F64 && prec != TMG_PREC_F32)) {
      c.err = "tmg_coarse_solve_noalloc: bad argument";
      return TMG_ERR_ARG;
    }
    if (!c.mg_ready) {
      c.err = "tmg_coarse_solve_noalloc: no setup";
      return TMG_ERR_STATE;
    }
    TMG_CUDA(cudaSetDevice(c.device));
    const size_t n = (size_t)c.cl.nc * c.cl.nd;
    const size_t es = prec == TMG_PREC_F64 ? sizeof(double2) : sizeof(float2);
    const size_t io = ((n * es + 255) & ~(size_t)255);
    const size_t need = 2 * io + tmg::coarse_gmres_scratch_bytes(c, prec);
    if (need > TMG_NOALLOC_SCRATCH_BYTES) {
      c.err = "tmg_coarse_solve_noalloc: the coarse problem needs " + std::to_string(need) +
              " bytes of scratch, more than the fixed " + std::to_string(TMG_NOALLOC_SCRATCH_BYTES) +
              " bytes; use tmg_coarse_solve";
      return TMG_ERR_ARG;
    }
    void* base = nullptr;
    const int rc = scratch_address(c.device, &base);
    if (rc != TMG_OK) {
      c.err = "tmg_coarse_solve_noalloc: cudaGetSymbolAddress failed";
      return rc;
    }
    char* s = (char*)base;
    void* bi = s;
    void* xo = s + io;
    void* work = s + 2 * io;
    const int grid = (int)std::min<size_t>((n + 255) / 256, (size_t)c.sms * 8);
    if (prec == TMG_PREC_F64) {
      TMG_CUDA(cudaMemcpyAsync(bi, b, n * sizeof(double2), cudaMemcpyDeviceToDevice, c.stream));
    } else {
      ++c.launches;
      k_noalloc_convert<<<grid, 256, 0, c.stream>>>((const double2*)b, (float2*)bi, n);
      TMG_CUDA(cudaGetLastError());
    }
    tmg::coarse_gmres_on_scratch(c, prec, bi, xo, mu, work);
    if (prec == TMG_PREC_F64) {
      TMG_CUDA(cudaMemcpyAsync(x, xo, n * sizeof(double2), cudaMemcpyDeviceToDevice, c.stream));
    } else {
      ++c.launches;
      k_noalloc_convert<<<grid, 256, 0, c.stream>>>((const float2*)xo, (double2*)x, n);
      TMG_CUDA(cudaGetLastError());
    }
    return TMG_OK;
  } catch (const tmg::Error& e) {
    c.err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    c.err = "tmg_coarse_solve_noalloc: host allocation failed";
    return TMG_ERR_OOM;
  } catch (const std::exception& e) {
    c.err = std::string("tmg_coarse_solve_noalloc: ") + e.what();
    return TMG_ERR_CUDA;
  }
}
