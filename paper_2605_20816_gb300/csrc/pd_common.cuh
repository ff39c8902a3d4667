// pd_common.cuh -- shared device-side building blocks of libpd:
// the multi-index set A_d, pixel coordinates, in-register Legendre features
// and the arithmetic traits of the FP64 / FP32 evaluation modes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "pd.h"

namespace pd {

// ---------------------------------------------------------------------------
// A_d in library order: ascending total degree, then descending alpha_1, then
// descending alpha_2 (Sec. 3.1 leaves the order to the implementation).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int basis_K(int dim, int d) {
  return dim == 2 ? (d + 1) * (d + 2) / 2 : (d + 1) * (d + 2) * (d + 3) / 6;
}

// Exponent of axis `ax` in the k-th multi-index.  Called with compile-time
// arguments inside unrolled loops, so it folds to a constant.
__host__ __device__ constexpr int basis_exp(int dim, int d, int k, int ax) {
  int idx = 0;
  for (int g = 0; g <= d; ++g) {
    if (dim == 2) {
      for (int a1 = g; a1 >= 0; --a1) {
        if (idx == k) return ax == 0 ? a1 : (ax == 1 ? g - a1 : 0);
        ++idx;
      }
    } else {
      for (int a1 = g; a1 >= 0; --a1)
        for (int a2 = g - a1; a2 >= 0; --a2) {
          if (idx == k) return ax == 0 ? a1 : (ax == 1 ? a2 : g - a1 - a2);
          ++idx;
        }
    }
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Pixel set.  Structured grid centres x_a = -1 + (2 k_a + 1) / n_a (Sec. 2.1)
// or an explicit point list.
// ---------------------------------------------------------------------------
struct Geom {
  int64_t n0, n1, n2;
  const double* coords;  // device [P][dim] or nullptr
  int64_t P;
};

template <int DIM, typename T>
__device__ __forceinline__ void pixel_coords(const Geom& g, int64_t j, T* x) {
  if (g.coords) {
#pragma unroll
    for (int a = 0; a < DIM; ++a) x[a] = (T)g.coords[j * DIM + a];
    return;
  }
  int64_t k0 = j % g.n0;
  int64_t r = j / g.n0;
  x[0] = (T)(-1.0 + (2.0 * (double)k0 + 1.0) / (double)g.n0);
  if (DIM == 2) {
    x[1] = (T)(-1.0 + (2.0 * (double)r + 1.0) / (double)g.n1);
  } else {
    int64_t k1 = r % g.n1;
    int64_t k2 = r / g.n1;
    x[1] = (T)(-1.0 + (2.0 * (double)k1 + 1.0) / (double)g.n1);
    x[2] = (T)(-1.0 + (2.0 * (double)k2 + 1.0) / (double)g.n2);
  }
}

// Tensor-product Legendre features psi_alpha(x) = prod_a P_{alpha_a}(x_a)
// (eq. h-degree-d-legendre), with P_m from the three-term recurrence
// (m+1) P_{m+1} = (2m+1) t P_m - m P_{m-1}, all in registers.  The
// multi-index of every output is a template constant, so the per-axis
// tables are indexed statically and stay in registers.
template <int DIM, int D, int k, typename T>
__device__ __forceinline__ T basis_product(const T (&Pm)[DIM][D + 1]) {
  constexpr int e0 = basis_exp(DIM, D, k, 0);
  constexpr int e1 = basis_exp(DIM, D, k, 1);
  constexpr int e2 = basis_exp(DIM, D, k, 2);
  T v = (T)1 * Pm[0][e0];
  v = v * Pm[1][e1];
  if constexpr (DIM == 3) v = v * Pm[2][e2];
  return v;
}

template <int DIM, int D, typename T, int... Ks>
__device__ __forceinline__ void basis_all(const T (&Pm)[DIM][D + 1], T* eta,
                                          std::integer_sequence<int, Ks...>) {
  ((eta[Ks] = basis_product<DIM, D, Ks>(Pm)), ...);
}

template <int DIM, int D, typename T>
__device__ __forceinline__ void legendre_features(const T* x, T* eta) {
  T Pm[DIM][D + 1];
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    Pm[a][0] = (T)1;
    if (D >= 1) Pm[a][1] = x[a];
#pragma unroll
    for (int m = 1; m < D; ++m)
      Pm[a][m + 1] = ((T)(2 * m + 1) * x[a] * Pm[a][m] - (T)m * Pm[a][m - 1]) / (T)(m + 1);
  }
  basis_all<DIM, D>(Pm, eta, std::make_integer_sequence<int, basis_K(DIM, D)>{});
}

// ---------------------------------------------------------------------------
// Arithmetic of the evaluation modes.
// FP64: logits in natural units, l_i = theta_i . eta * (-1/eps), exp/log.
// FP32: logits in base-2 units, l_i = theta_i . eta * (-log2(e)/eps), so
//       the soft assignment is one MUFU ex2 per pixel-grain pair.
// ---------------------------------------------------------------------------
template <typename T>
struct Arith;

template <>
struct Arith<double> {
  static __device__ __forceinline__ double ex(double v) { return exp(v); }
  static __device__ __forceinline__ double lg(double v) { return log(v); }
  static constexpr double to_nat = 1.0;  // logit units -> natural log
  static double theta_scale(double eps) { return -1.0 / eps; }
};

template <>
struct Arith<float> {
  static __device__ __forceinline__ float ex(float v) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
  }
  static __device__ __forceinline__ float lg(float v) {
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
  }
  static constexpr double to_nat = 0.693147180559945309417232121458176568;  // ln 2
  static double theta_scale(double eps) { return -1.4426950408889634073599246810018921 / eps; }
};

// The log-sum-exp of a pixel whose label term is kept apart (log2 units):
// m the running max (m >= lG), s the sum of 2^(l_k - m) over the grains
// other than the label G, lG the label's logit.  With rho = s 2^(m - lG),
// p_G = 1 / (1 + rho), so
//   log2 S = lG + log2(1 + rho),  1 - p_G = rho / (1 + rho),
//   log p_G = -log(1 + rho),
// none of which cancels when p_G is close to 1 (rho small).  Below
// p_G = 2^-100 nothing cancels and S is taken directly.  A NaN lG (a label
// outside 0..N-1) gives log2 S from s and a NaN log p_G.
struct LabelLse {
  float lse, q;
  double logp;
};
__device__ __forceinline__ LabelLse label_lse(float m, float s, float lG) {
  LabelLse r;
  if (lG - m >= -100.f) {
    const float rho = __fdividef(s, Arith<float>::ex(lG - m));
    const float l1 = log1pf(rho);
    r.lse = fmaf(l1, 1.44269504088896341f, lG);
    r.q = __fdividef(rho, 1.f + rho);
    r.logp = -(double)l1;
  } else {
    r.lse = m + log2f(s);
    r.q = 1.f;
    r.logp = (double)(lG - r.lse) * Arith<float>::to_nat;
  }
  return r;
}

// Row stride of the scaled parameter copy: K padded to a 16-byte multiple.
template <typename T>
__host__ __device__ constexpr int padded_K(int K) {
  return sizeof(T) == 4 ? (K + 3) / 4 * 4 : (K + 1) / 2 * 2;
}

}  // namespace pd
