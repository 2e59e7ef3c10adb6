// noalloc.cu -- second-order energy of a context without any device allocation.
//
// pnm_mbpt2 keeps its per-row partial sums in memory the context allocated.  Some callers
// cannot allocate device memory at the point where they want the number: real-time or
// embedded loops whose device-memory budget is fixed when they start (an allocation later
// can fail or stall them), and hosts whose device allocator belongs to another framework
// that forbids side allocations.  pnm_mbpt2_noalloc serves them: its scratch is the
// file-scope array below, which every GPU that loads this library holds until the process
// exits.
#include <mutex>
#include <new>

#include "pnm_context.cuh"

// Partial sums (one per (channel, ij) row) followed by one result per system.
#define PNM_NOALLOC_MAX_ROWS 65536
#define PNM_NOALLOC_MAX_SYSTEMS 64
#define PNM_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_mbpt2_scratch[PNM_NOALLOC_MAX_ROWS + PNM_NOALLOC_MAX_SYSTEMS];

// Device address of g_mbpt2_scratch per device.  In host code the array's name is only a
// host-side stand-in, so the address is looked up once per device with that device current
// (by the first call on that device).  The cached address is valid for the life of the
// device's primary context: a cudaDeviceReset in between would leave it stale.
static std::mutex g_scratch_mu;
static double* g_scratch_addr[PNM_NOALLOC_MAX_DEVICES] = {};

static double* scratch_on(int dev) {
  if (dev < 0 || dev >= PNM_NOALLOC_MAX_DEVICES) throw PnmError{PNM_EINVAL, "device index out of range"};
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    int prev = 0;
    CUDA_TRY(cudaGetDevice(&prev));
    if (prev != dev) CUDA_TRY(cudaSetDevice(dev));
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_mbpt2_scratch);
    if (prev != dev) cudaSetDevice(prev);
    if (e != cudaSuccess)
      throw PnmError{PNM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e)};
    g_scratch_addr[dev] = (double*)p;
  }
  return g_scratch_addr[dev];
}

extern "C" int pnm_mbpt2_noalloc(const pnm_ctx* ctx, double* dE) {
  // every failure becomes a status code: nothing may leave an extern "C" function as an
  // exception (the mutex, the message strings and the CUDA calls can all throw)
  try {
    if (!ctx || !dE) throw PnmError{PNM_EINVAL, "null argument"};
    int nsys = (int)ctx->sys.size();
    if (ctx->nrows > PNM_NOALLOC_MAX_ROWS)
      throw PnmError{PNM_EINVAL, "context has " + std::to_string(ctx->nrows) +
                                     " (channel, hole-pair) rows; pnm_mbpt2_noalloc handles at most " +
                                     std::to_string(PNM_NOALLOC_MAX_ROWS)};
    if (nsys > PNM_NOALLOC_MAX_SYSTEMS)
      throw PnmError{PNM_EINVAL, "pnm_mbpt2_noalloc handles at most " +
                                     std::to_string(PNM_NOALLOC_MAX_SYSTEMS) + " systems"};
    int dev = 0;
    CUDA_TRY(cudaStreamGetDevice(ctx->stream, &dev));
    double* scratch = scratch_on(dev);
    // every partial and result slot used here is written before it is read: nothing to clear
    pnm_launch_mbpt2_into(ctx, scratch, scratch + PNM_NOALLOC_MAX_ROWS);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(dE, scratch + PNM_NOALLOC_MAX_ROWS, sizeof(double) * nsys,
                             cudaMemcpyDeviceToHost, ctx->stream));
    CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return PNM_OK;
  } catch (const PnmError& e) {
    pnm_set_error(e.code, e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    pnm_set_error(PNM_ENOMEM, "host allocation failed");
    return PNM_ENOMEM;
  } catch (...) {
    pnm_set_error(PNM_EINVAL, "unexpected failure");
    return PNM_EINVAL;
  }
}
