// Waveform post-processing of the Psi4 modes (Sec. 2.3 of the SACRA-K paper):
// Nakano's extrapolation to infinity with the retarded time, and the fixed
// frequency integration of Psi4 to the strain.  Device arrays of the caller,
// no device allocation by this library; the FFTs are cuFFT's, loaded at the
// first call (only these entry points depend on it) and run on the caller's
// work area.
#include <dlfcn.h>

#include <cmath>
#include <cufft.h>
#include <mutex>

#include "../../include/sacrak.h"
#include "sacrak_dev.cuh"

namespace sacrak {

constexpr int NK_THREADS = 1024;

// One block: the trapezoid time integral as a fixed-order chunked scan (each
// thread sums its chunk of increments, thread 0 scans the chunk totals in
// order, each thread rewalks its chunk from its offset), then
// out = C (D0 psi - (l-1)(l+2)/2 int) and t_ret = t - shift.
__global__ void __launch_bounds__(NK_THREADS) nakano_kernel(const double* __restrict__ t,
                                                            const double2* __restrict__ psi, int n,
                                                            double d0, double c, double coef, double shift,
                                                            double* __restrict__ t_ret,
                                                            double2* __restrict__ out) {
  __shared__ double2 off[NK_THREADS];
  const int chunk = (n + NK_THREADS - 1) / NK_THREADS;
  const int lo = threadIdx.x * chunk, hi = min(n, lo + chunk);
  double2 s = make_double2(0.0, 0.0);
  for (int i = max(lo, 1); i < hi; ++i) {
    const double h = 0.5 * (t[i] - t[i - 1]);
    s.x += h * (psi[i].x + psi[i - 1].x);
    s.y += h * (psi[i].y + psi[i - 1].y);
  }
  off[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 run = make_double2(0.0, 0.0);
    for (int k = 0; k < NK_THREADS; ++k) {
      const double2 v = off[k];
      off[k] = run;
      run.x += v.x;
      run.y += v.y;
    }
  }
  __syncthreads();
  double2 run = off[threadIdx.x];
  for (int i = lo; i < hi; ++i) {
    if (i > 0) {
      const double h = 0.5 * (t[i] - t[i - 1]);
      run.x += h * (psi[i].x + psi[i - 1].x);
      run.y += h * (psi[i].y + psi[i - 1].y);
    }
    out[i] = make_double2(c * (d0 * psi[i].x - coef * run.x), c * (d0 * psi[i].y - coef * run.y));
    t_ret[i] = t[i] - shift;
  }
}

// h_k <- h_k / (2 pi max(|f_k|, f_cut))^2 / n over the DFT frequencies
// f_k = k / (n dt) for k < (n+1)/2, (k - n) / (n dt) otherwise
__global__ void ffi_scale_kernel(double2* h, int n, double dt, double f_cut) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double f = (k < (n + 1) / 2 ? (double)k : (double)(k - n)) / (n * dt);
  const double a = 2.0 * 3.141592653589793 * fmax(fabs(f), f_cut);
  const double s = 1.0 / (a * a * n);
  h[k] = make_double2(h[k].x * s, h[k].y * s);
}

namespace {

struct Cufft {
  cufftResult (*create)(cufftHandle*);
  cufftResult (*set_auto)(cufftHandle, int);
  cufftResult (*make1d)(cufftHandle, int, cufftType, int, size_t*);
  cufftResult (*set_work)(cufftHandle, void*);
  cufftResult (*set_stream)(cufftHandle, cudaStream_t);
  cufftResult (*exec)(cufftHandle, cufftDoubleComplex*, cufftDoubleComplex*, int);
  cufftResult (*destroy)(cufftHandle);
  bool ok = false;
};

const Cufft& cufft() {
  static Cufft f;
  static std::once_flag once;
  std::call_once(once, [] {
    void* h = nullptr;
    for (const char* name : {"libcufft.so.12", "libcufft.so", "/usr/local/cuda/lib64/libcufft.so.12",
                             "/usr/local/cuda/lib64/libcufft.so"})
      if (!h) h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
    if (!h) return;
    f.create = (decltype(f.create))dlsym(h, "cufftCreate");
    f.set_auto = (decltype(f.set_auto))dlsym(h, "cufftSetAutoAllocation");
    f.make1d = (decltype(f.make1d))dlsym(h, "cufftMakePlan1d");
    f.set_work = (decltype(f.set_work))dlsym(h, "cufftSetWorkArea");
    f.set_stream = (decltype(f.set_stream))dlsym(h, "cufftSetStream");
    f.exec = (decltype(f.exec))dlsym(h, "cufftExecZ2Z");
    f.destroy = (decltype(f.destroy))dlsym(h, "cufftDestroy");
    f.ok = f.create && f.set_auto && f.make1d && f.set_work && f.set_stream && f.exec && f.destroy;
  });
  return f;
}

// a Z2Z plan of length n without an automatic work area; its size in *ws
bool make_plan(int n, cufftHandle* plan, size_t* ws) {
  const Cufft& F = cufft();
  if (!F.ok || F.create(plan) != CUFFT_SUCCESS) return false;
  if (F.set_auto(*plan, 0) != CUFFT_SUCCESS || F.make1d(*plan, n, CUFFT_Z2Z, 1, ws) != CUFFT_SUCCESS) {
    F.destroy(*plan);
    return false;
  }
  return true;
}

}  // namespace
}  // namespace sacrak

using namespace sacrak;

extern "C" {

sacrak_status sacrak_nakano(const double* t, const double* psi, int n, int l, double r0, double m0,
                            double* t_ret, double* out, void* cuda_stream) {
  if (!t || !psi || !t_ret || !out || n < 1 || l < 2 || !(r0 > 0.0) || !(m0 > 0.0) || !std::isfinite(r0) ||
      !std::isfinite(m0))
    return SACRAK_EINVAL;
  const double d0 = r0 * (1.0 + m0 / (2.0 * r0)) * (1.0 + m0 / (2.0 * r0));
  if (!(d0 / (2.0 * m0) > 1.0)) return SACRAK_EINVAL;  // the logarithm of t_ret
  const double c = 1.0 - 2.0 * m0 / d0;
  const double shift = d0 + 2.0 * m0 * std::log(d0 / (2.0 * m0) - 1.0);
  const double coef = 0.5 * (l - 1) * (l + 2);
  nakano_kernel<<<1, NK_THREADS, 0, (cudaStream_t)cuda_stream>>>(t, (const double2*)psi, n, d0, c, coef, shift,
                                                                  t_ret, (double2*)out);
  return cudaGetLastError() == cudaSuccess ? SACRAK_OK : SACRAK_ECUDA;
}

size_t sacrak_ffi_work_bytes(int n) {
  if (n < 1) return 0;
  cufftHandle plan;
  size_t ws = 0;
  if (!make_plan(n, &plan, &ws)) return 0;
  cufft().destroy(plan);
  return ws > 0 ? ws : 1;
}

sacrak_status sacrak_ffi_strain(const double* psi, int n, double dt, double f_cut, double* h, void* work,
                                size_t work_bytes, void* cuda_stream) {
  if (!psi || !h || n < 1 || !(dt > 0.0) || !(f_cut > 0.0) || !std::isfinite(dt) || !std::isfinite(f_cut))
    return SACRAK_EINVAL;
  cufftHandle plan;
  size_t ws = 0;
  if (!make_plan(n, &plan, &ws)) return SACRAK_ECUDA;
  const Cufft& F = cufft();
  sacrak_status st = SACRAK_OK;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (ws > work_bytes || (ws > 0 && !work)) {
    st = SACRAK_EINVAL;
  } else if (F.set_work(plan, work) != CUFFT_SUCCESS || F.set_stream(plan, s) != CUFFT_SUCCESS) {
    st = SACRAK_ECUDA;
  } else if (cudaMemcpyAsync(h, psi, sizeof(double) * 2 * n, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
    st = SACRAK_ECUDA;
  } else if (F.exec(plan, (cufftDoubleComplex*)h, (cufftDoubleComplex*)h, CUFFT_FORWARD) != CUFFT_SUCCESS) {
    st = SACRAK_ECUDA;
  } else {
    ffi_scale_kernel<<<(n + 255) / 256, 256, 0, s>>>((double2*)h, n, dt, f_cut);
    if (cudaGetLastError() != cudaSuccess ||
        F.exec(plan, (cufftDoubleComplex*)h, (cufftDoubleComplex*)h, CUFFT_INVERSE) != CUFFT_SUCCESS)
      st = SACRAK_ECUDA;
  }
  // the plan is destroyed after the work queued on the stream that uses it
  if (cudaStreamSynchronize(s) != cudaSuccess) st = SACRAK_ECUDA;
  F.destroy(plan);
  return st;
}

}  // extern "C"
