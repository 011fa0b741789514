// Host-side operator generator (long double); see opgen.h.
#include "opgen.h"

#include <cmath>
#include <cstring>

namespace sesc {
namespace {

typedef long double ld;

// Legendre polynomial P_k(x) and its derivative by the three-term recurrence.
void legendre(int k, ld x, ld* p, ld* dp) {
  ld p0 = 1.0L, p1 = x;
  if (k == 0) { *p = 1.0L; *dp = 0.0L; return; }
  for (int j = 2; j <= k; ++j) {
    ld p2 = ((2 * j - 1) * x * p1 - (j - 1) * p0) / j;
    p0 = p1;
    p1 = p2;
  }
  *p = p1;
  *dp = k * (x * p1 - p0) / (x * x - 1.0L);
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration from Chebyshev guesses.
void gauss_legendre(int n, ld* x, ld* w) {
  const ld pi = 3.14159265358979323846264338327950288L;
  for (int i = 0; i < n; ++i) {
    ld z = -cosl(pi * (i + 0.75L) / (n + 0.5L));
    for (int it = 0; it < 100; ++it) {
      ld p, dp;
      legendre(n, z, &p, &dp);
      ld dz = p / dp;
      z -= dz;
      if (fabsl(dz) < 1e-30L) break;
    }
    ld p, dp;
    legendre(n, z, &p, &dp);
    x[i] = z;
    w[i] = 2.0L / ((1.0L - z * z) * dp * dp);
  }
}

// Gauss-Lobatto nodes/weights on [-1, 1]: end points and roots of P'_{n-1}.
void gauss_lobatto(int n, ld* x, ld* w) {
  const ld pi = 3.14159265358979323846264338327950288L;
  const int k = n - 1;
  for (int i = 0; i < n; ++i) {
    ld z = -cosl(pi * i / k);
    if (i > 0 && i < k) {
      for (int it = 0; it < 100; ++it) {
        // f = P_k'(z); f' = P_k''(z) = (2 z P_k' - k (k+1) P_k) / (1 - z^2)
        ld p, dp;
        legendre(k, z, &p, &dp);
        ld d2 = (2.0L * z * dp - k * (k + 1) * p) / (1.0L - z * z);
        ld dz = dp / d2;
        z -= dz;
        if (fabsl(dz) < 1e-30L) break;
      }
    }
    ld p, dp;
    if (i == 0 || i == k) {
      p = (i == 0 && (k % 2)) ? -1.0L : 1.0L;
    } else {
      legendre(k, z, &p, &dp);
    }
    x[i] = z;
    w[i] = 2.0L / (k * (k + 1) * p * p);
  }
}

// Barycentric weights of the nodes.
void bary_weights(int n, const ld* x, ld* bw) {
  for (int j = 0; j < n; ++j) {
    ld prod = 1.0L;
    for (int k = 0; k < n; ++k)
      if (k != j) prod *= (x[j] - x[k]);
    bw[j] = 1.0L / prod;
  }
}

// Values l_j(y) of all Lagrange polynomials at y (barycentric form).
void lagrange_at(int n, const ld* x, const ld* bw, ld y, ld* out) {
  for (int j = 0; j < n; ++j)
    if (y == x[j]) {
      for (int k = 0; k < n; ++k) out[k] = (k == j) ? 1.0L : 0.0L;
      return;
    }
  ld den = 0.0L;
  for (int j = 0; j < n; ++j) den += bw[j] / (y - x[j]);
  for (int j = 0; j < n; ++j) out[j] = bw[j] / (y - x[j]) / den;
}

// In-place inverse of an n x n matrix by Gauss-Jordan elimination with pivoting.
bool invert(int n, ld* A) {
  ld aug[8][16];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < 2 * n; ++j) aug[i][j] = (j < n) ? A[i * n + j] : ((j - n) == i ? 1.0L : 0.0L);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabsl(aug[r][c]) > fabsl(aug[piv][c])) piv = r;
    if (aug[piv][c] == 0.0L) return false;
    if (piv != c)
      for (int j = 0; j < 2 * n; ++j) { ld tmp = aug[c][j]; aug[c][j] = aug[piv][j]; aug[piv][j] = tmp; }
    ld d = aug[c][c];
    for (int j = 0; j < 2 * n; ++j) aug[c][j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      ld f = aug[r][c];
      for (int j = 0; j < 2 * n; ++j) aug[r][j] -= f * aug[c][j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[i * n + j] = aug[i][n + j];
  return true;
}

}  // namespace

bool make_level_ops(int n, int family, LevelOps* out) {
  if (!(n == 2 || n == 4 || n == 8) || !(family == 0 || family == 1) || out == nullptr) return false;
  std::memset(out, 0, sizeof(LevelOps));
  out->n = n;
  ld x[8], w[8], bw[8];
  if (family == 0) gauss_legendre(n, x, w); else gauss_lobatto(n, x, w);
  for (int i = 0; i < n; ++i) { x[i] *= 0.5L; w[i] *= 0.5L; }   // map to [-1/2, 1/2], sum 1
  bary_weights(n, x, bw);

  // nodal differentiation matrix, barycentric formula
  ld D[64];
  for (int i = 0; i < n; ++i) {
    ld diag = 0.0L;
    for (int j = 0; j < n; ++j) {
      if (i == j) continue;
      D[i * n + j] = (bw[j] / bw[i]) / (x[i] - x[j]);
      diag -= D[i * n + j];
    }
    D[i * n + i] = diag;
  }
  // projection: P_ij = n * integral of l_j over subcell i, n-point Gauss rule per subcell
  ld gx[8], gw[8];
  gauss_legendre(n, gx, gw);
  ld P[64] = {0};
  ld val[8];
  for (int i = 0; i < n; ++i) {
    ld a = -0.5L + (ld)i / n, b = a + 1.0L / n;
    for (int q = 0; q < n; ++q) {
      ld y = 0.5L * (a + b) + 0.5L * (b - a) * gx[q];
      lagrange_at(n, x, bw, y, val);
      for (int j = 0; j < n; ++j) P[i * n + j] += n * 0.5L * (b - a) * gw[q] * val[j];
    }
  }
  ld R[64];
  std::memcpy(R, P, sizeof(R));
  if (!invert(n, R)) return false;
  // Dvol = M^-1 D^T M, Dhat = P Dvol
  ld Dvol[64], Dhat[64];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Dvol[i * n + j] = w[j] * D[j * n + i] / w[i];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      ld s = 0.0L;
      for (int k = 0; k < n; ++k) s += P[i * n + k] * Dvol[k * n + j];
      Dhat[i * n + j] = s;
    }
  // boundary columns of Bsurf = M^-1 B: -l_i(-1/2)/w_i and l_i(1/2)/w_i; Bhat = P B^(0)
  ld lm[8], lp[8];
  lagrange_at(n, x, bw, -0.5L, lm);
  lagrange_at(n, x, bw, 0.5L, lp);
  ld Bh0[8], Bhn[8];
  for (int i = 0; i < n; ++i) {
    ld s0 = 0.0L, sn = 0.0L;
    for (int k = 0; k < n; ++k) {
      s0 += P[i * n + k] * (-lm[k] / w[k]);
      sn += P[i * n + k] * (lp[k] / w[k]);
    }
    Bh0[i] = s0;
    Bhn[i] = sn;
    out->Bh0[i] = (double)s0;
    out->Bhn[i] = (double)sn;
  }
  // telescoping form: cumulative sums over the first k rows
  for (int k = 1; k < n; ++k) {
    ld a0 = 0.0L, an = 0.0L;
    for (int i = 0; i < k; ++i) { a0 += Bh0[i]; an += Bhn[i]; }
    out->c0[k - 1] = (double)(1.0L + a0 / n);
    out->cn[k - 1] = (double)(an / n);
    for (int j = 0; j < n; ++j) {
      ld c = 0.0L;
      for (int i = 0; i < k; ++i) c += Dhat[i * n + j];
      out->C[(k - 1) * n + j] = (double)c;
    }
  }
  // interface values from means: IRf = I_face R, I_face[k][j] = l_j(-1/2 + k/n)
  for (int k = 0; k <= n; ++k) {
    lagrange_at(n, x, bw, -0.5L + (ld)k / n, val);
    for (int j = 0; j < n; ++j) {
      ld s = 0.0L;
      for (int m = 0; m < n; ++m) s += val[m] * R[m * n + j];
      out->IRf[k * n + j] = (double)s;
    }
  }
  for (int i = 0; i < n * n; ++i) {
    out->R[i] = (double)R[i];
    out->P[i] = (double)P[i];
    out->Dn[i] = (double)D[i];
    out->Dhat[i] = (double)Dhat[i];
  }
  for (int i = 0; i < n; ++i) { out->w[i] = (double)w[i]; out->nodes[i] = (double)x[i]; }
  return true;
}

}  // namespace sesc
