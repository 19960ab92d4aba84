// Complex arithmetic on CUDA's float2 / double2 (x = real part, y = imaginary part), usable in
// host and device code.
#pragma once
#include <cuda_runtime.h>

namespace icwf {

template <typename T> struct cplx;
template <> struct cplx<double> { using type = double2; };
template <> struct cplx<float> { using type = float2; };
template <typename T> using c_t = typename cplx<T>::type;

template <typename T> __host__ __device__ __forceinline__ c_t<T> mk(T re, T im) {
  c_t<T> z; z.x = re; z.y = im; return z;
}
template <typename Z> __host__ __device__ __forceinline__ Z cadd(Z a, Z b) { a.x += b.x; a.y += b.y; return a; }
template <typename Z> __host__ __device__ __forceinline__ Z csub(Z a, Z b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename Z> __host__ __device__ __forceinline__ Z cmul(Z a, Z b) {
  Z r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// conj(a) * b
template <typename Z> __host__ __device__ __forceinline__ Z cmulc(Z a, Z b) {
  Z r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
template <typename Z> __host__ __device__ __forceinline__ Z cconj(Z a) { a.y = -a.y; return a; }
template <typename Z, typename S> __host__ __device__ __forceinline__ Z cscale(Z a, S s) { a.x *= s; a.y *= s; return a; }

}  // namespace icwf
