// icwf_observables_static: the observables of icwf_observables computed without allocating any
// device memory during the call.
//
// Who needs it: hosts whose allocator policy forbids device allocation once they have started,
// e.g. an application that reserves its device memory in one arena at start-up and treats any
// later cudaMalloc as a fault, or a deployment that must not allocate on its serving path.
// icwf_observables allocates its work buffers (the wavefunction on the full grid and the reduction
// partials) on its first call; this entry point uses one fixed work area compiled into the library
// instead.  The call copies its results into the caller's (pageable) host arrays and waits for its
// stream, so it must run outside any stream capture.
//
// The work area is a file-scope static device array of ICWF_OBS_STATIC_BYTES bytes; every GPU
// that loads the library holds it until the process exits.  Host code cannot use the array's name
// as a device address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (with that device current) and caches it.  All calls share the one work
// area: calls that overlap on the GPU race, so the caller serialises them.  Each call writes every
// part of the work area that it later reads, so nothing carried over from an earlier call needs
// clearing.
#include <cuda_runtime.h>

#include <mutex>

#include "icwf_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_obs_work[ICWF_OBS_STATIC_BYTES];

constexpr int kMaxDevices = 64;
void* g_addr[kMaxDevices] = {nullptr};
std::mutex g_mutex;

size_t up256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of the work area on `device` (looked up once per device).
cudaError_t work_area(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  if (g_addr[device]) {
    *out = g_addr[device];
    return cudaSuccess;
  }
  int prev = 0;
  cudaError_t e = cudaGetDevice(&prev);
  if (e != cudaSuccess) return e;
  if (prev != device && (e = cudaSetDevice(device)) != cudaSuccess) return e;
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_obs_work);
  if (prev != device) cudaSetDevice(prev);
  if (e != cudaSuccess) return e;
  g_addr[device] = p;
  *out = p;
  return cudaSuccess;
}

}  // namespace

extern "C" icwf_status icwf_observables_static(icwf_handle h, icwf_obs* out) {
  using namespace icwf;
  ObsView v;
  if (!h || !handle_obs_view(h, &v)) {
    handle_set_error(nullptr, "icwf_observables_static: NULL handle");
    return ICWF_ERR_ARG;
  }
  if (!out) {
    handle_set_error(h, "icwf_observables_static: out is NULL");
    return ICWF_ERR_ARG;
  }
  if (!v.initialised) {
    handle_set_error(h, "icwf_observables_static: handle not initialised");
    return ICWF_ERR_STATE;
  }
  const int nx = v.j.nx, nR = v.j.nR;
  if ((size_t)nx * nR > ICWF_OBS_STATIC_MAX_GRID || nx > 4096 || nR > 4096) {
    handle_set_error(h, "icwf_observables_static: grid too large for the static work area "
                        "(nx * nR must be <= 524288)");
    return ICWF_ERR_ARG;
  }
  // carve the work area
  const size_t need = up256((size_t)nx * nR * sizeof(double2)) + up256((size_t)nx * 8) +
                      up256((size_t)nR * 8) + up256((size_t)(2 * nR + nx) * 8) + up256(64 * 8) +
                      up256(8 * 8) + up256(64 * 8) + up256((size_t)8 * nR * sizeof(double2));
  if (need > ICWF_OBS_STATIC_BYTES) {
    handle_set_error(h, "icwf_observables_static: work area too small for this grid");
    return ICWF_ERR_ARG;
  }
  void* base = nullptr;
  cudaError_t e = work_area(v.device, &base);
  if (e != cudaSuccess) {
    handle_set_error(h, "icwf_observables_static: cudaGetSymbolAddress failed");
    return ICWF_ERR_CUDA;
  }
  char* p = (char*)base;
  auto take = [&](size_t b) { char* q = p; p += up256(b); return (void*)q; };
  double2* Psi = (double2*)take((size_t)nx * nR * sizeof(double2));
  double* rho_x = (double*)take((size_t)nx * 8);
  double* rho_R = (double*)take((size_t)nR * 8);
  double* part = (double*)take((size_t)(2 * nR + nx) * 8);
  double* o4 = (double*)take(64 * 8);
  double* pop = (double*)take(8 * 8);
  double* decoh = (double*)take(64 * 8);
  double2* proj = (double2*)take((size_t)8 * nR * sizeof(double2));

  cudaStream_t s = v.stream;
  if (v.mixed) launch_reconstruct<float>(v.j, v.C, Psi, s);
  else launch_reconstruct<double>(v.j, v.C, Psi, s);
  launch_obs_lines(v.j, Psi, v.phi, v.n_states, rho_x, rho_R, proj, part, o4, pop, decoh,
                   v.twx_d, v.twR_d, s);
  // a launch error of these kernels is reported without clearing errors left by other callers
  if (cudaPeekAtLastError() != cudaSuccess) {
    handle_set_error(h, "icwf_observables_static: kernel launch failed");
    return ICWF_ERR_CUDA;
  }
  double host4[4];
  int cl[2];
  bool ok = cudaMemcpyAsync(host4, o4, sizeof(host4), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
            cudaMemcpyAsync(cl, v.j.status, sizeof(cl), cudaMemcpyDeviceToHost, s) == cudaSuccess;
  if (ok && out->rho_x)
    ok = cudaMemcpyAsync(out->rho_x, rho_x, (size_t)nx * 8, cudaMemcpyDeviceToHost, s) == cudaSuccess;
  if (ok && out->rho_R)
    ok = cudaMemcpyAsync(out->rho_R, rho_R, (size_t)nR * 8, cudaMemcpyDeviceToHost, s) == cudaSuccess;
  if (ok && out->pop && v.n_states)
    ok = cudaMemcpyAsync(out->pop, pop, (size_t)v.n_states * 8, cudaMemcpyDeviceToHost, s) == cudaSuccess;
  if (ok && out->decoh && v.n_states)
    ok = cudaMemcpyAsync(out->decoh, decoh, (size_t)v.n_states * v.n_states * 8,
                         cudaMemcpyDeviceToHost, s) == cudaSuccess;
  if (ok) ok = cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    handle_set_error(h, "icwf_observables_static: a CUDA call failed");
    return ICWF_ERR_CUDA;
  }
  out->t = v.t;
  out->norm = host4[0];
  out->energy = (host4[1] + host4[2] + host4[3]) / host4[0];
  out->n_states = v.n_states;
  out->n_clamped = cl[1];
  return ICWF_OK;
}
