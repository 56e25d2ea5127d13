// kbc_common.cuh -- lattice and storage traits shared by the CUDA kernels.
//
// Lattices D2Q9 / D3Q27 are tensor products of D1Q3 (weights 2/3 for c = 0,
// 1/6 for c = +-1).  Direction index i = (cz+1)*9 + (cy+1)*3 + (cx+1)
// (D2Q9: i = (cy+1)*3 + (cx+1)); the opposite direction is Q-1-i.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace kbc {

template <int Q>
struct Lat;

template <>
struct Lat<9> {
  static constexpr int Q = 9, D = 2;
  __host__ __device__ static constexpr int cx(int i) { return i % 3 - 1; }
  __host__ __device__ static constexpr int cy(int i) { return i / 3 - 1; }
  __host__ __device__ static constexpr int cz(int) { return 0; }
};

template <>
struct Lat<27> {
  static constexpr int Q = 27, D = 3;
  __host__ __device__ static constexpr int cx(int i) { return i % 3 - 1; }
  __host__ __device__ static constexpr int cy(int i) { return (i / 3) % 3 - 1; }
  __host__ __device__ static constexpr int cz(int i) { return i / 9 - 1; }
};

__host__ __device__ constexpr double w1d(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }

template <class L>
__host__ __device__ constexpr double weight(int i) {
  return L::D == 2 ? w1d(L::cx(i)) * w1d(L::cy(i))
                   : w1d(L::cx(i)) * w1d(L::cy(i)) * w1d(L::cz(i));
}

// ---- storage of one population ------------------------------------------
// F32 keeps g = f - W; F16 / BF16 / F16N keep h = f/W - 1 so that every
// direction uses the full mantissa around O(u) deviations.
// F64 keeps g = f - W in double precision and computes in FP64 (the test
// storage: the FP32-compute path's reference on the GPU).
enum { STORE_F32 = 0, STORE_F16 = 1, STORE_BF16 = 2, STORE_F64 = 3, STORE_F16N = 4 };

template <int S>
struct Store;

template <>
struct Store<STORE_F32> {
  using C = float;  // compute type
  using T = float;
  static constexpr int bytes = 4;
  __device__ __forceinline__ static float load(const T *p, float /*w*/) { return __ldg(p); }
  __device__ __forceinline__ static float load_smem(const T *p, float /*w*/) { return *p; }
  __device__ __forceinline__ static void store(T *p, float g, float /*invw*/) { *p = g; }
  __device__ __forceinline__ static T encode(double g, double /*w*/) { return (float)g; }
  __device__ __forceinline__ static double decode(T v, double /*w*/) { return (double)v; }
  // two neighbouring values (8-byte aligned pair)
  __device__ __forceinline__ static float2 load2(const T *p, float /*w*/) {
    return __ldg(reinterpret_cast<const float2 *>(p));
  }
  __device__ __forceinline__ static void store2(T *p, float2 g, float /*invw*/) {
    *reinterpret_cast<float2 *>(p) = g;
  }
};

template <>
struct Store<STORE_F16> {
  using C = float;  // compute type
  using T = __half;
  static constexpr int bytes = 2;
  __device__ __forceinline__ static float load(const T *p, float w) {
    return w * __half2float(__ldg(p));
  }
  __device__ __forceinline__ static float load_smem(const T *p, float w) {
    return w * __half2float(*p);
  }
  __device__ __forceinline__ static void store(T *p, float g, float invw) {
    *p = __float2half_rn(g * invw);
  }
  __device__ __forceinline__ static T encode(double g, double w) { return __double2half(g / w); }
  __device__ __forceinline__ static double decode(T v, double w) {
    return w * (double)__half2float(v);
  }
  __device__ __forceinline__ static float2 load2(const T *p, float w) {
    const float2 h = __half22float2(__ldg(reinterpret_cast<const __half2 *>(p)));
    return __fmul2_rn(h, make_float2(w, w));
  }

  __device__ __forceinline__ static void store2(T *p, float2 g, float invw) {
    *reinterpret_cast<__half2 *>(p) = __float22half2_rn(__fmul2_rn(g, make_float2(invw, invw)));
  }
};

template <>
struct Store<STORE_BF16> {
  using C = float;  // compute type
  using T = __nv_bfloat16;
  static constexpr int bytes = 2;
  __device__ __forceinline__ static float load(const T *p, float w) {
    return w * __bfloat162float(__ldg(p));
  }
  __device__ __forceinline__ static float load_smem(const T *p, float w) {
    return w * __bfloat162float(*p);
  }
  __device__ __forceinline__ static void store(T *p, float g, float invw) {
    *p = __float2bfloat16_rn(g * invw);
  }
  __device__ __forceinline__ static T encode(double g, double w) {
    return __float2bfloat16_rn((float)(g / w));
  }
  __device__ __forceinline__ static double decode(T v, double w) {
    return w * (double)__bfloat162float(v);
  }
  __device__ __forceinline__ static float2 load2(const T *p, float w) {
    const float2 h = __bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162 *>(p)));
    return __fmul2_rn(h, make_float2(w, w));
  }

  __device__ __forceinline__ static void store2(T *p, float2 g, float invw) {
    *reinterpret_cast<__nv_bfloat162 *>(p) =
        __float22bfloat162_rn(__fmul2_rn(g, make_float2(invw, invw)));
  }
};

template <>
struct Store<STORE_F64> {
  using T = double;
  using C = double;  // compute type
  static constexpr int bytes = 8;
  __device__ __forceinline__ static double load(const T *p, double /*w*/) { return __ldg(p); }
  __device__ __forceinline__ static void store(T *p, double g, double /*invw*/) { *p = g; }
  __device__ __forceinline__ static T encode(double g, double /*w*/) { return g; }
  __device__ __forceinline__ static double decode(T v, double /*w*/) { return v; }
};

// F16N: a 16-bit float of h = f/W - 1 with its exponent range narrowed to
// what h needs: sign, 3 exponent bits, 12 stored significand bits.  Codes
// e = 1..7 hold (1 + m/4096) 2^(e-7), |h| in [2^-6, 2); e = 0 holds m 2^-18
// (evenly spaced below 2^-6).  Against IEEE half (5 exponent bits, 10 stored
// significand bits) the step is four times finer wherever |h| >= 2^-6, which
// covers the O(u) deviations of the moving populations; |h| >= 2 saturates
// at the largest code (h is below 1.4 for |u| <= 0.1).
// The 15 magnitude bits shifted left by 11 are the FP32 bit pattern of
// |h| 2^-120 (codes e = 0 land on FP32 subnormals, which keep their exact
// value: no flush-to-zero in this build), so decoding is two shifts, one
// logic operation and the multiply by W 2^120; encoding is the multiply by
// 2^-120 / W, rounding the 11 dropped bits to nearest (ties away from zero)
// with an integer add that carries into the exponent, and a saturating min.
template <>
struct Store<STORE_F16N> {
  using C = float;  // compute type
  using T = uint16_t;
  static constexpr int bytes = 2;
  __device__ __forceinline__ static float bits_to_scaled(uint32_t c) {
    return __uint_as_float(((c & 0x8000u) << 16) | ((c & 0x7FFFu) << 11));  // |h| 2^-120, signed
  }
  __device__ __forceinline__ static uint16_t scaled_to_bits(float x) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t a = min((b & 0x7FFFFFFFu) + 0x400u, 0x3FFFFFFu);
    return (uint16_t)(((b >> 16) & 0x8000u) | (a >> 11));
  }
  __device__ __forceinline__ static float load(const T *p, float w) {
    return bits_to_scaled(__ldg(p)) * (w * 0x1p120f);
  }
  __device__ __forceinline__ static float load_smem(const T *p, float w) {
    return bits_to_scaled(*p) * (w * 0x1p120f);
  }
  __device__ __forceinline__ static void store(T *p, float g, float invw) {
    *p = scaled_to_bits(g * (invw * 0x1p-120f));
  }
  __device__ __forceinline__ static T encode(double g, double w) {
    return scaled_to_bits((float)(g / w * 0x1p-120));
  }
  __device__ __forceinline__ static double decode(T v, double w) {
    return w * 0x1p120 * (double)bits_to_scaled(v);
  }
  __device__ __forceinline__ static float2 load2(const T *p, float w) {
    const uint32_t c = __ldg(reinterpret_cast<const unsigned int *>(p));
    const float2 x = make_float2(bits_to_scaled(c & 0xFFFFu), bits_to_scaled(c >> 16));
    const float s = w * 0x1p120f;
    return __fmul2_rn(x, make_float2(s, s));
  }
  __device__ __forceinline__ static void store2(T *p, float2 g, float invw) {
    const float s = invw * 0x1p-120f;
    const float2 x = __fmul2_rn(g, make_float2(s, s));
    *reinterpret_cast<unsigned int *>(p) =
        (uint32_t)scaled_to_bits(x.x) | ((uint32_t)scaled_to_bits(x.y) << 16);
  }
};

// Node flags (one byte per stored node, ghosts included).
enum : uint8_t { NODE_FLUID = 0, NODE_SOLID = 1, NODE_GHOST = 3 };

// Geometry of the stored lattice: interior nx*ny*nz, padded by one ghost
// layer on every non-periodic axis.
struct Grid {
  int nx, ny, nz;     // interior
  int NX, NY, NZ;     // stored (interior + ghosts)
  int px, py, pz;     // ghost padding per axis (0 periodic, 1 otherwise)
  int pitch;          // row stride in elements: NX rounded up to a multiple of 8
                      // (every row starts on a 16-byte boundary for bulk copies)
  long long N;        // pitch*NY*NZ, the population plane stride
};

__host__ __device__ __forceinline__ long long sidx(const Grid &g, int X, int Y, int Z) {
  return ((long long)Z * g.NY + Y) * g.pitch + X;
}

// Neighbour coordinate in stored space: wraps only on periodic axes (a padded
// axis keeps X-1 >= 0 and X+1 < NX for every interior node).
__device__ __forceinline__ int nbr(int X, int c, int NX) {
  int s = X + c;
  if (s < 0) s += NX;
  if (s >= NX) s -= NX;
  return s;
}

}  // namespace kbc
