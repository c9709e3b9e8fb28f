// CPU oracle of the CGLS solve, matrix-free, complex128, OpenMP.
//
// TEST INFRASTRUCTURE ONLY: the timed CPU baseline of bench.py and its pins in tests/ load it;
// the product path never does, and it shares no code with the CUDA path.  It restates, as plain
// loops over the grid, the same definitions as oracle/wri_oracle.py:
//   * the operator of the paper's Sec. "3D Source free WRI" (A = omega^2 diag(m) + Laplacian)
//     with the stretched-coordinate absorbing layer of our reading:
//       (A u)_n = omega^2 w_n m_n u_n + sum over axes [c(+1/2) (u_next - u_n) - c(-1/2) (u_n - u_prev)],
//       c^x(i +- 1/2) = s_y(j) s_z(k) / (s_x(i +- 1/2) h^2) (likewise y, z), w = s_x s_y s_z,
//       s(xi) = 1 + i sigma(xi)/omega, sigma = sigma_max (xi/L)^2, sigma_max = 3 v_max ln(1/R)/(2L),
//       u = 0 outside the grid;
//   * A^H by its definition, (A^H y)_n = sum over rows r of conj(A_rn) y_r: the coefficient
//     of node n in a neighbour's row, conjugated (no use of A's symmetry);
//   * S = [Z A ; lambda P] (Z = I - e e^H in source-free mode, I otherwise), b = [b1 ; lambda d]
//     (Eqs. CmpctWRIobj / Sandb, lambda on the data term);
//   * CGLS (Algorithm 1 read as CGLS): t = S p, alpha = gamma / ||t||^2, x += alpha p,
//     r -= alpha t, s = S^H r, gamma' = ||s||^2, stop when sqrt(gamma') <= tol ||S^H b||,
//     beta = gamma' / gamma, p = s + beta p; x0 = 0.
#include <cmath>
#include <complex>
#include <cstdint>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

typedef std::complex<double> cd;

// stretch factors of one axis at the nodes (pos = i) and at the half points (pos = i - 1/2,
// i = 0..n, so half[i] lies between nodes i-1 and i)
void stretch(int n, int npml, double h, double omega, double v_max, double R, std::vector<cd>& node,
             std::vector<cd>& half) {
  auto s_of = [&](double pos) -> cd {
    if (npml <= 0) return cd(1.0, 0.0);
    const double L = npml * h;
    const double smax = 3.0 * v_max * std::log(1.0 / R) / (2.0 * L);
    double xi = 0.0;
    if (pos < npml) xi = (npml - pos) * h;
    else if (pos > n - 1 - npml) xi = (pos - (n - 1 - npml)) * h;
    const double sigma = smax * (xi / L) * (xi / L);
    return cd(1.0, sigma / omega);
  };
  node.resize(n);
  half.resize(n + 1);
  for (int i = 0; i < n; ++i) node[i] = s_of(i);
  for (int i = 0; i <= n; ++i) half[i] = s_of(i - 0.5);
}

struct Helmholtz {
  int nx, ny, nz;
  long long n;
  double om2;
  const double* m;
  std::vector<cd> sx, sy, sz;     // node stretch factors
  std::vector<cd> ix, iy, iz;     // 1 / (s(half point) h^2); entry i is the half point i - 1/2

  long long idx(int i, int j, int k) const { return ((long long)k * ny + j) * nx + i; }

  // entries of row (i, j, k): the six neighbour coefficients and the centre
  cd xm(int i, int j, int k) const { return sy[j] * sz[k] * ix[i]; }
  cd xp(int i, int j, int k) const { return sy[j] * sz[k] * ix[i + 1]; }
  cd ym(int i, int j, int k) const { return sx[i] * sz[k] * iy[j]; }
  cd yp(int i, int j, int k) const { return sx[i] * sz[k] * iy[j + 1]; }
  cd zm(int i, int j, int k) const { return sx[i] * sy[j] * iz[k]; }
  cd zp(int i, int j, int k) const { return sx[i] * sy[j] * iz[k + 1]; }
  cd centre(int i, int j, int k) const {
    return om2 * (sx[i] * sy[j] * sz[k]) * m[idx(i, j, k)] -
           (xm(i, j, k) + xp(i, j, k) + ym(i, j, k) + yp(i, j, k) + zm(i, j, k) + zp(i, j, k));
  }

  // y = A x
  void apply(const cd* x, cd* y) const {
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          cd v = centre(i, j, k) * x[idx(i, j, k)];
          if (i > 0) v += xm(i, j, k) * x[idx(i - 1, j, k)];
          if (i < nx - 1) v += xp(i, j, k) * x[idx(i + 1, j, k)];
          if (j > 0) v += ym(i, j, k) * x[idx(i, j - 1, k)];
          if (j < ny - 1) v += yp(i, j, k) * x[idx(i, j + 1, k)];
          if (k > 0) v += zm(i, j, k) * x[idx(i, j, k - 1)];
          if (k < nz - 1) v += zp(i, j, k) * x[idx(i, j, k + 1)];
          y[idx(i, j, k)] = v;
        }
  }

  // y = A^H x: node n collects conj(A_rn) x_r from its own row and from the rows of its six
  // neighbours, in each of which n is the opposite neighbour
  void apply_adjoint(const cd* x, cd* y) const {
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
          cd v = std::conj(centre(i, j, k)) * x[idx(i, j, k)];
          if (i > 0) v += std::conj(xp(i - 1, j, k)) * x[idx(i - 1, j, k)];
          if (i < nx - 1) v += std::conj(xm(i + 1, j, k)) * x[idx(i + 1, j, k)];
          if (j > 0) v += std::conj(yp(i, j - 1, k)) * x[idx(i, j - 1, k)];
          if (j < ny - 1) v += std::conj(ym(i, j + 1, k)) * x[idx(i, j + 1, k)];
          if (k > 0) v += std::conj(zp(i, j, k - 1)) * x[idx(i, j, k - 1)];
          if (k < nz - 1) v += std::conj(zm(i, j, k + 1)) * x[idx(i, j, k + 1)];
          y[idx(i, j, k)] = v;
        }
  }
};

// 1 / (s h^2) at every half point of an axis
std::vector<cd> inverse_half(const std::vector<cd>& half, double h) {
  std::vector<cd> out(half.size());
  for (size_t i = 0; i < half.size(); ++i) out[i] = 1.0 / (half[i] * (h * h));
  return out;
}

double norm2(const std::vector<cd>& v) {
  double s = 0.0;
  const long long n = (long long)v.size();
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (long long e = 0; e < n; ++e) s += std::norm(v[e]);
  return s;
}

}  // namespace

extern "C" {

// One CGLS solve of min ||S x - b|| for one system (see the header comment).
//   grid: nx, ny, nz (computational nodes), npml, h, omega, pml_R, v_max
//   m [n] squared slowness; src node; source_free 1 (Z applied, b1 = 0) or 0 (b1 = alpha e);
//   alpha [2] (re, im) when source_free = 0; rec [nrec] receiver nodes, d [2 nrec] data (re, im);
//   max_iter iterations at most, tol on ||S^H r|| / ||S^H b||; threads (0 = OpenMP default).
//   Out: x [2 n] (re, im), *iters, *relres.  Returns 0, or 1 on an invalid argument.
int oracle_cgls(int nx, int ny, int nz, int npml, double h, double omega, double pml_R, double v_max,
                const double* m, long long src, int source_free, const double* alpha, int nrec, const int* rec,
                const double* d, double lam, int max_iter, double tol, int threads, double* x_out, int* iters,
                double* relres) {
  if (nx < 1 || ny < 1 || nz < 1 || !m || !x_out || !iters || !relres || max_iter < 0 || (nrec > 0 && (!rec || !d)))
    return 1;
  const long long n = (long long)nx * ny * nz;
  if (src < 0 || src >= n || (!source_free && !alpha)) return 1;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#else
  (void)threads;
#endif
  Helmholtz A;
  A.nx = nx;
  A.ny = ny;
  A.nz = nz;
  A.n = n;
  A.om2 = omega * omega;
  A.m = m;
  std::vector<cd> hx, hy, hz;
  stretch(nx, npml, h, omega, v_max, pml_R, A.sx, hx);
  stretch(ny, npml, h, omega, v_max, pml_R, A.sy, hy);
  stretch(nz, npml, h, omega, v_max, pml_R, A.sz, hz);
  A.ix = inverse_half(hx, h);
  A.iy = inverse_half(hy, h);
  A.iz = inverse_half(hz, h);

  // t = S v: t1 = Z A v (n), t2 = lambda P v (nrec)
  auto S = [&](const std::vector<cd>& v, std::vector<cd>& t1, std::vector<cd>& t2) {
    A.apply(v.data(), t1.data());
    if (source_free) t1[src] = 0.0;
    for (int q = 0; q < nrec; ++q) t2[q] = lam * v[rec[q]];
  };
  // s = S^H (r1, r2) = A^H Z r1 + lambda P^T r2 (Z is real and diagonal)
  std::vector<cd> zr(n);
  auto SH = [&](const std::vector<cd>& r1, const std::vector<cd>& r2, std::vector<cd>& s) {
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n; ++e) zr[e] = r1[e];
    if (source_free) zr[src] = 0.0;
    A.apply_adjoint(zr.data(), s.data());
    for (int q = 0; q < nrec; ++q) s[rec[q]] += lam * r2[q];
  };

  std::vector<cd> x(n, 0.0), r1(n, 0.0), r2(nrec), s(n), p(n), t1(n), t2(nrec);
  if (!source_free) r1[src] = cd(alpha[0], alpha[1]);
  for (int q = 0; q < nrec; ++q) r2[q] = lam * cd(d[2 * q], d[2 * q + 1]);
  SH(r1, r2, s);  // x0 = 0: r = b, s = S^H b
  const double ref = std::sqrt(norm2(s));
  double gamma = norm2(s);
  p = s;
  int it = 0;
  double rr = ref > 0 ? std::sqrt(gamma) / ref : 0.0;
  while (it < max_iter && rr > tol) {
    S(p, t1, t2);
    double delta = norm2(t1);
    for (int q = 0; q < nrec; ++q) delta += std::norm(t2[q]);
    const double al = gamma / delta;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n; ++e) {
      x[e] += al * p[e];
      r1[e] -= al * t1[e];
    }
    for (int q = 0; q < nrec; ++q) r2[q] -= al * t2[q];
    SH(r1, r2, s);
    const double gnew = norm2(s);
    ++it;
    rr = std::sqrt(gnew) / ref;
    if (rr <= tol) break;
    const double beta = gnew / gamma;
    gamma = gnew;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < n; ++e) p[e] = s[e] + beta * p[e];
  }
  for (long long e = 0; e < n; ++e) {
    x_out[2 * e] = x[e].real();
    x_out[2 * e + 1] = x[e].imag();
  }
  *iters = it;
  *relres = rr;
  return 0;
}

// Threads an OpenMP parallel region of this library runs with.
int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"
