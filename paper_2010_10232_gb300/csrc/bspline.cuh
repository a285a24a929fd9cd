// Device-side B-spline evaluation shared by the setup and load kernels
// (Section 2.3.1: Cox-de Boor recursion on an open knot vector).
#pragma once
#include "common.cuh"

// Gauss-Legendre node i (ascending) and weight of the n-point rule on [-1, 1]:
// Newton's method on the three-term Legendre recurrence from the Chebyshev-like
// starting value, nodes mirrored so the rule is exactly symmetric.
__device__ inline void gauss_node(int n, int i, double* xo, double* wo) {
  int ii = (i < n / 2) ? i : n - 1 - i;
  double x = -cos(3.14159265358979323846 * (ii + 0.75) / (n + 0.5));
  double dp = 1.0;
  for (int it = 0; it < 60; ++it) {
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (x * p1 - p0) / (x * x - 1.0);
    double dx = p1 / dp;
    x -= dx;
    if (fabs(dx) < 1e-17) break;
  }
  {
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = (n == 1) ? 1.0 : n * (x * p1 - p0) / (x * x - 1.0);
  }
  double w = 2.0 / ((1.0 - x * x) * dp * dp);
  if ((n & 1) && ii == n / 2) x = 0.0;
  if (i != ii) x = -x;
  *xo = x;
  *wo = w;
}

// Values v[a] = phi_{s-p+a, p}(x) and derivatives d[a] of the p+1 B-splines that
// are active on knot span s (t[s] <= x < t[s+1]), by the Cox-de Boor recursion.
__device__ inline void active_basis(const double* t, int p, int s, double x, double* v, double* d) {
  double cur[IGA_MAXP + 1], nxt[IGA_MAXP + 1];
  cur[0] = 1.0;
  for (int q = 1; q <= p; ++q) {
    if (q == p) {   // derivatives from the degree p-1 values
      for (int a = 0; a <= p; ++a) {
        int j = s - p + a;
        double r = 0.0;
        if (a - 1 >= 0) {
          double d1 = t[j + p] - t[j];
          if (d1 != 0.0) r += p / d1 * cur[a - 1];
        }
        if (a <= p - 1) {
          double d2 = t[j + p + 1] - t[j + 1];
          if (d2 != 0.0) r -= p / d2 * cur[a];
        }
        d[a] = r;
      }
    }
    for (int a = 0; a <= q; ++a) {
      int j = s - q + a;
      double term = 0.0;
      if (a - 1 >= 0) {
        double d1 = t[j + q] - t[j];
        if (d1 != 0.0) term += (x - t[j]) / d1 * cur[a - 1];
      }
      if (a <= q - 1) {
        double d2 = t[j + q + 1] - t[j + 1];
        if (d2 != 0.0) term += (t[j + q + 1] - x) / d2 * cur[a];
      }
      nxt[a] = term;
    }
    for (int a = 0; a <= q; ++a) cur[a] = nxt[a];
  }
  for (int a = 0; a <= p; ++a) v[a] = cur[a];
  if (p == 0) d[0] = 0.0;
}


// Knot span s in [p, n_el+p-1] with t[s] <= x < t[s+1]; the right end point
// belongs to the last span.
__device__ inline int find_span(const double* t, int n_el, int p, double x) {
  int lo = p, hi = n_el + p - 1;
  if (x >= t[hi]) return hi;
  while (lo < hi) {
    int mid = (lo + hi + 1) / 2;
    if (t[mid] <= x) lo = mid; else hi = mid - 1;
  }
  return lo;
}
