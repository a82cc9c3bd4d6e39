// k_noalloc.cu -- dlr_sweep_noalloc: the sweep entry point for callers that
// must not allocate device memory.  Its scratch (the directions, the edge
// inflow values and the bounded-wait flag) lives in one fixed-size array in
// this file instead of stream-ordered allocations.
#include <cuda_runtime.h>

#include "../../include/dlr.h"
#include "dlr_internal.cuh"

namespace dlr {
template <typename real>
cudaError_t launch_sweep_dirs(int, int, double, double, int, const double *, const double *,
                              const real *, const real *, real *, int *, cudaStream_t);
int record_error(int code, const char *msg);  // message for dlr_last_error()
int sweep_width_check(int nx, int ny, int precision);  // DLR_EINVAL for a mesh too wide
}

namespace {

// Layout (doubles): [0, 2*MAX) directions, [2*MAX, 2*MAX+4) edge inflow,
// then one int (the wait flag).  Every GPU that loads the library holds
// this array until the process exits.
constexpr int kMaxDirs = DLR_SWEEP_NOALLOC_MAX_DIRS;
constexpr int kScratchDoubles = 2 * kMaxDirs + 4 + 4;
__device__ __align__(256) double g_sweep_scratch[kScratchDoubles];

int err(int code, const char *m) { return dlr::record_error(code, m); }

}  // namespace

extern "C" int dlr_sweep_noalloc(int32_t nx, int32_t ny, double lx, double ly, int32_t n_dir,
                                 const double *dirs, const double *psi_edge, int32_t precision,
                                 const void *sigma_t, const void *src, void *psi, void *stream) {
  if (nx < 1 || ny < 1 || n_dir < 1 || !dirs || !psi_edge || !sigma_t || !src || !psi ||
      !(lx > 0) || !(ly > 0) || (precision != DLR_FP64 && precision != DLR_MIXED))
    return err(DLR_EINVAL, "bad argument to dlr_sweep_noalloc");
  if (n_dir > kMaxDirs) return err(DLR_EINVAL, "n_dir exceeds DLR_SWEEP_NOALLOC_MAX_DIRS");
  // the same mesh-width limit as dlr_sweep, checked before anything is enqueued
  if (int rc = dlr::sweep_width_check(nx, ny, precision)) return rc;
  // The device address of the array on the current device.  In host code
  // the array's name is only a host-side stand-in, not a device address, so
  // it is looked up on every call (cheap, allocates nothing, and never stale
  // after a context teardown); the first lookup on a device may load the
  // library's device code there, so make the first call before any stream
  // capture.
  void *addr = nullptr;
  {
    cudaError_t e = cudaGetSymbolAddress(&addr, g_sweep_scratch);
    if (e != cudaSuccess || !addr) {
      cudaGetLastError();
      return err(DLR_ECUDA, cudaGetErrorString(e));
    }
  }
  double *base = static_cast<double *>(addr);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double *d_dirs = base;
  double *d_edge = base + 2 * kMaxDirs;
  int *d_wait = reinterpret_cast<int *>(base + 2 * kMaxDirs + 4);
  cudaError_t e = cudaMemcpyAsync(d_dirs, dirs, sizeof(double) * 2 * n_dir, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_edge, psi_edge, sizeof(double) * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_wait, 0, sizeof(int), st);  // the flag must start at zero
  if (e != cudaSuccess) return err(DLR_ECUDA, cudaGetErrorString(e));
  const double hx = lx / nx, hy = ly / ny;
  e = precision == DLR_MIXED
          ? dlr::launch_sweep_dirs<float>(nx, ny, hx, hy, n_dir, d_dirs, d_edge,
                                          static_cast<const float *>(sigma_t),
                                          static_cast<const float *>(src), static_cast<float *>(psi),
                                          d_wait, st)
          : dlr::launch_sweep_dirs<double>(nx, ny, hx, hy, n_dir, d_dirs, d_edge,
                                           static_cast<const double *>(sigma_t),
                                           static_cast<const double *>(src),
                                           static_cast<double *>(psi), d_wait, st);
  if (e != cudaSuccess) return err(DLR_ECUDA, cudaGetErrorString(e));
  int waited_out = 0;
  e = cudaMemcpyAsync(&waited_out, d_wait, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return err(DLR_ECUDA, cudaGetErrorString(e));
  if (waited_out) return err(DLR_ETIMEOUT, "a sweep wait timed out");
  return DLR_OK;
}
