// Stolt source coordinate of the f-k temporal stage (Sec. 4.2, Alg. 1,
// Listing 2) in float-float arithmetic: mu = sqrt(A + m^2) with A from
// float64 per-plan tables split into (hi, lo) floats, m^2 exact, and one
// Newton correction of the square root from an exact FMA residual. Plain
// float would put the interpolation weight off by up to 6e-5 near m ~ 1000.
#pragma once
#include <cuda_runtime.h>

namespace nlos {

__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return make_float2(s, (a - (s - bb)) + (b - bb));
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return make_float2(s, b - (s - a));
}

struct StoltCoord {
  int k0, k1;
  float alpha, jac;
  bool valid;
};

// mu = sqrt(A + m^2) to ~1e-11 absolute: y0 = S * rsqrt(S) is within a few
// ulp of sqrt(S); one Newton step from the exact FMA residual S - y0^2 gives
// mu = y0 + mlo. The weight m/mu uses the same reciprocal square root.
__device__ __forceinline__ StoltCoord stolt_coord(float Ahi, float Alo, int m, int n) {
  StoltCoord c;
  float2 s = two_sum(Ahi, (float)(m * m));
  s = fast_two_sum(s.x, s.y + Alo);
  const float rs = rsqrtf(s.x);
  const float y0 = s.x * rs;
  const float res = fmaf(-y0, y0, s.x) + s.y;     // (A + m^2) - y0^2
  const float mlo = res * (0.5f * rs);            // mu = y0 + mlo
  int k0 = (int)floorf(y0);
  float al = (y0 - (float)k0) + mlo;
  if (al < 0.f) {
    k0 -= 1;
    al += 1.f;
  } else if (al >= 1.f) {
    k0 += 1;
    al -= 1.f;
  }
  c.valid = (k0 < n - 1) || (k0 == n - 1 && al == 0.f);
  c.k0 = k0;
  c.k1 = min(k0 + 1, n - 1);
  c.alpha = al;
  c.jac = (float)m * rs;
  return c;
}

// The same coordinate from a per-pencil split of A into an integer and a
// fraction: S = A + m^2 = (Ai + m^2) + Af, where Ai + m^2 is an exact integer
// (below 2^24 wherever the source can lie in a spectrum: mu < L/2 <= 4096)
// and Af = A - Ai in [0, 1] is one float (absolute error <= 2^-25, so mu to
// about 1.5e-8 / mu). S then takes one exact sum instead of two, and the
// weight's rollover at an integer one floor instead of two branches.
struct StoltSplitA {
  int Ai;
  float Af;
};
__device__ __forceinline__ StoltSplitA stolt_split_a(float Ahi, float Alo) {
  // sources with A >= 2^24 lie outside every spectrum: A is clamped to
  // exactly 2^24 (and the sum stays positive and in range); so is a NaN
  if (!(Ahi < 16777216.f)) return {16777216, 0.f};
  const int Ai = (int)Ahi;   // floor: A >= 0; Ahi - Ai is exact
  return {Ai, (Ahi - (float)Ai) + Alo};
}
// m >= 1, fm = (float)m
__device__ __forceinline__ StoltCoord stolt_coord_split(const StoltSplitA& a, int m, float fm, int n) {
  StoltCoord c;
  const float sx = (float)(a.Ai + m * m);
  const float sh = sx + a.Af;                 // |sx| >= 1 >= |Af|: fast two-sum
  const float sl = a.Af - (sh - sx);
  const float rs = rsqrtf(sh);
  const float y0 = sh * rs;
  const float res = fmaf(-y0, y0, sh) + sl;   // S - y0^2
  const float mlo = res * (0.5f * rs);        // mu = y0 + mlo
  int k0 = (int)floorf(y0);
  float al = (y0 - (float)k0) + mlo;
  const float roll = floorf(al);              // -1, 0 or 1: y0 is within a few ulp of mu
  k0 += (int)roll;
  al -= roll;
  c.valid = (k0 < n - 1) || (k0 == n - 1 && al == 0.f);
  c.k0 = k0;
  c.k1 = k0 + 1;
  c.alpha = al;
  c.jac = fm * rs;
  return c;
}

}  // namespace nlos
