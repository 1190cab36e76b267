// CPU oracle of PCG-ATKM (Tang, Wang, Zhang & Zhang, "An efficient and
// accurate numerical method for computing the ground states of
// three-dimensional rotating dipolar Bose-Einstein condensates under strongly
// anisotropic trap"): TEST INFRASTRUCTURE ONLY.
//
// A plain, slow restatement of the paper's method in C++17 and binary64, with
// its own FFT.  It is loaded only by the tests, by the smoke check and by the
// CPU-baseline leg of the benchmark; the product path never calls it, and it
// shares no code, header, table or constant generator with the CUDA library.
// Every step follows the paper in its order and notation; there is no
// blocking, fusion or reordering beyond the definitions below.  OpenMP runs
// independent FFT lines and independent grid planes in parallel; every sum is
// taken in a fixed order (per z-plane, then over the planes in order), so the
// results do not depend on the number of threads.
//
// Arrays are row-major [N_z][N_y][N_x] (x fastest); complex values are
// interleaved (re, im) binary64 pairs.
//
// Readings of the paper where it is silent or garbled (the same readings as
// the solver's; each is also listed in the design notes):
//   * truncated-kernel coefficients: the unshifted real even
//     U0(nu) = int_{D_2L} e^{-i nu.y} / (4 pi |y|) dy (Eq. (FUk) without the
//     basis phase (-1)^{k_x+k_y+k_z}); rho occupies padded indices [0, N)
//     and the result is cropped to [0, N); the output is real-part'ed;
//   * the kernel in g_n of Eq. (Energy_Expend) is U_dip;
//   * stop rule ||H phi - mu phi|| <= tol (or ||phi_{n+1} - phi_n||_inf, Eq.
//     (stop_maxnorm)); "halve until the energy decreases" accepts
//     E+ <= E + 32 eps |E|, at most max_halvings halvings, then the lowest
//     trial is taken and the next direction is steepest descent; three
//     consecutive exhausted loops end the run as stagnated;
//   * phi is divided by its norm after each retraction; a Step 4 reset p is
//     the p_n kept for the next Polak-Ribiere step.
#include <stdint.h>

#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

const double kPi = 3.14159265358979323846264338327950288;

// ---------------------------------------------------------------- complex
struct cx {
  double re, im;
};
inline cx cadd(cx a, cx b) { return {a.re + b.re, a.im + b.im}; }
inline cx csub(cx a, cx b) { return {a.re - b.re, a.im - b.im}; }
inline cx cmul(cx a, cx b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
inline cx cscale(cx a, double s) { return {a.re * s, a.im * s}; }
inline cx cdiv(cx a, cx b) {
  // Smith's algorithm (R. L. Smith, CACM 5, 1962): no overflow for large |b|
  if (std::fabs(b.re) >= std::fabs(b.im)) {
    const double r = b.im / b.re, d = b.re + b.im * r;
    return {(a.re + a.im * r) / d, (a.im - a.re * r) / d};
  }
  const double r = b.re / b.im, d = b.re * r + b.im;
  return {(a.re * r + a.im) / d, (a.im * r - a.re) / d};
}
inline cx cexp(cx a) {
  const double m = std::exp(a.re);
  return {m * std::cos(a.im), m * std::sin(a.im)};
}

// ---------------------------------------------------------------- FFT
// Discrete Fourier transform of one length n (§2.1, Eq. (FourphiCo) is
// this DFT scaled by 1/n): y_k = sum_j x_j exp(sign 2 pi i j k / n).
// Recursive decimation in time: n = p m with p the smallest prime factor of
// n; the p interleaved subsequences x_{p j + r} are transformed (length m)
// and combined, X_{k + q m} = sum_r W_p^{r q} (W_n^{r k} Y_r[k]).  Any n
// works; lengths whose factors are 2, 3 and 5 recurse down to 2-, 3- and
// 5-point DFTs.
struct Dft {
  int n = 0;
  std::vector<cx> root[2];  // root[0][j] = exp(-2 pi i j / n), root[1][j] = its conjugate

  explicit Dft(int len) : n(len) {
    root[0].resize(len);
    root[1].resize(len);
    for (int j = 0; j < len; ++j) {
      const double th = 2.0 * kPi * (double)j / (double)len;
      root[0][j] = {std::cos(th), -std::sin(th)};
      root[1][j] = {std::cos(th), std::sin(th)};
    }
  }
  static int smallest_factor(int m) {
    for (int p = 2; p * p <= m; ++p)
      if (m % p == 0) return p;
    return m;
  }
  // y[0..len) = DFT_len of x[0], x[s], ..., x[(len-1) s]; `step` = n / len
  // maps the length-len roots W_len^e = tw[e step] onto the table.  x and y
  // must not overlap.
  void rec(const cx* x, long s, cx* y, int len, long step, const cx* tw) const {
    if (len == 1) {
      y[0] = x[0];
      return;
    }
    const int p = smallest_factor(len);
    const int m = len / p;
    for (int r = 0; r < p; ++r) rec(x + r * s, s * p, y + (long)r * m, m, step * p, tw);
    if (p == 2) {  // X_k = Y_0[k] + W^k Y_1[k], X_{k+m} = Y_0[k] - W^k Y_1[k]
      for (int k = 0; k < m; ++k) {
        const cx a = y[k], b = cmul(y[m + k], tw[(long)k * step]);
        y[k] = cadd(a, b);
        y[m + k] = csub(a, b);
      }
      return;
    }
    cx tb[8], ub[8];
    std::vector<cx> tv, uv;
    cx *t = tb, *u = ub;
    if (p > 8) {
      tv.resize(p);
      uv.resize(p);
      t = tv.data();
      u = uv.data();
    }
    for (int k = 0; k < m; ++k) {
      t[0] = y[k];
      for (int r = 1; r < p; ++r) t[r] = cmul(y[(long)r * m + k], tw[(long)r * k * step]);
      for (int q = 0; q < p; ++q) {
        cx acc = t[0];
        for (int r = 1; r < p; ++r) acc = cadd(acc, cmul(t[r], tw[(long)((r * q) % p) * m * step]));
        u[q] = acc;
      }
      for (int q = 0; q < p; ++q) y[(long)q * m + k] = u[q];
    }
  }
  void apply(const cx* x, cx* y, int sign) const { rec(x, 1, y, n, 1, root[sign > 0 ? 1 : 0].data()); }
};

// In-place 3D DFT of a [nz][ny][nx] array along x, then y, then z.
// sign = -1: forward, scaled by 1/(nx ny nz) (the coefficients of Eq.
// (FourphiCo)); sign = +1: the unscaled sum over the coefficients (Eq.
// (Fourphi) at the grid points).
void fft3(cx* a, int nx, int ny, int nz, int sign, const Dft& Dx, const Dft& Dy, const Dft& Dz, int threads) {
  const int mx = nx > ny ? (nx > nz ? nx : nz) : (ny > nz ? ny : nz);
#pragma omp parallel num_threads(threads)
  {
    std::vector<cx> bi(mx), bo(mx);
#pragma omp for schedule(static)
    for (long line = 0; line < (long)ny * nz; ++line) {
      cx* row = a + line * nx;
      for (int i = 0; i < nx; ++i) bi[i] = row[i];
      Dx.apply(bi.data(), bo.data(), sign);
      for (int i = 0; i < nx; ++i) row[i] = bo[i];
    }
#pragma omp for schedule(static)
    for (long col = 0; col < (long)nx * nz; ++col) {
      const long z = col / nx, x = col % nx;
      cx* base = a + z * (long)ny * nx + x;
      for (int j = 0; j < ny; ++j) bi[j] = base[(long)j * nx];
      Dy.apply(bi.data(), bo.data(), sign);
      for (int j = 0; j < ny; ++j) base[(long)j * nx] = bo[j];
    }
#pragma omp for schedule(static)
    for (long col = 0; col < (long)nx * ny; ++col) {
      cx* base = a + col;
      for (int k = 0; k < nz; ++k) bi[k] = base[(long)k * nx * ny];
      Dz.apply(bi.data(), bo.data(), sign);
      for (int k = 0; k < nz; ++k) base[(long)k * nx * ny] = bo[k];
    }
    if (sign < 0) {
      const double sc = 1.0 / ((double)nx * ny * nz);
#pragma omp for schedule(static)
      for (long j = 0; j < (long)nx * ny * nz; ++j) a[j] = cscale(a[j], sc);
    }
  }
}

// ---------------------------------------------------------------- Faddeeva
// w(z) = e^{-z^2} erfc(-i z) for Im z > 0, written from two published
// methods:
//  * |z| <= 8: the trapezoidal rule for w(z) = (i/pi) int e^{-t^2}/(z - t) dt
//    with step h = 0.4 and the pole correction of Chiarella & Reichel (Math.
//    Comp. 22, 1968) and Matta & Reichel (Math. Comp. 25, 1971):
//    w(z) = (i h/pi) sum_n e^{-t_n^2}/(z - t_n) + 2 e^{-z^2}/(1 -/+ e^{-2 pi i z/h}),
//    nodes t_n = n h (sign -) or (n + 1/2) h (sign +), whichever keeps Re z
//    at least h/4 from every node; the neglected terms are O(e^{-pi^2/h^2});
//  * |z| > 8: the Laplace continued fraction
//    w(z) = (i/sqrt(pi)) / (z - (1/2)/(z - 1/(z - (3/2)/(z - ...)))),
//    60 levels, evaluated from the bottom.
cx faddeeva(cx z) {
  const double az = std::sqrt(z.re * z.re + z.im * z.im);
  if (az > 8.0) {
    cx t = z;
    for (int k = 60; k >= 1; --k) t = csub(z, cdiv(cx{0.5 * k, 0.0}, t));
    return cscale(cdiv(cx{0.0, 1.0}, t), 1.0 / std::sqrt(kPi));
  }
  const double h = 0.4;
  const int M = 18;  // e^{-(M h)^2} < 1e-22
  const double fr = z.re / h - std::floor(z.re / h);
  const double delta = (std::fabs(fr - 0.5) < 0.25) ? 0.0 : 0.5;
  cx sum = {0.0, 0.0};
  for (int n = -M; n <= M; ++n) {
    const double t = (n + delta) * h;
    sum = cadd(sum, cscale(cdiv(cx{1.0, 0.0}, cx{z.re - t, z.im}), std::exp(-t * t)));
  }
  const cx T = cmul(cx{0.0, h / kPi}, sum);
  // e^{-z^2} and e^{-2 pi i z / h}
  const cx ez = cexp(cx{-(z.re * z.re - z.im * z.im), -2.0 * z.re * z.im});
  const cx q = cexp(cx{2.0 * kPi * z.im / h, -2.0 * kPi * z.re / h});
  const cx den = delta == 0.0 ? cx{1.0 - q.re, -q.im} : cx{1.0 + q.re, q.im};
  return cadd(T, cdiv(cscale(ez, 2.0), den));
}

// I(s; nu) = int_{-a}^{a} e^{-s^2 y^2} cos(nu y) dy for nu = pi k / a:
// (sqrt(pi)/s) e^{-nu^2/4s^2} Re erf(s a + i nu/(2s))
//   = (sqrt(pi)/s) Re[e^{-nu^2/4s^2} - e^{-s^2 a^2} e^{-i nu a} w(-nu/(2s) + i s a)],
// e^{-i nu a} = (-1)^k; (sqrt(pi)/s) erf(s a) for k = 0.
double axis_integral(int k, double a, double s) {
  if (k == 0) return std::sqrt(kPi) / s * std::erf(s * a);
  const double nu = kPi * k / a;
  const cx w = faddeeva(cx{-nu / (2.0 * s), s * a});
  const double sg = (k % 2 == 0) ? 1.0 : -1.0;
  return std::sqrt(kPi) / s * (std::exp(-nu * nu / (4.0 * s * s)) - std::exp(-(s * a) * (s * a)) * sg * w.re);
}

// ---------------------------------------------------------------- plan
struct Grid {
  int N[3];
  double L[3], h[3], hvol;
  long n;
};

int kfreq(int m, int M) { return m < M / 2 ? m : m - M; }

struct Plan {
  Grid g;
  double dip[3];
  int threads;
  Dft *dx, *dy, *dz, *px, *py, *pz;
  std::vector<double> U0;  // [N_z+1][N_y+1][N_x+1], indexed by |k|
  std::vector<double> K;   // [2N_z][2N_y][2N_x], FFT order
  std::vector<double> xc, yc, zc, nux, nuy, nuz;
};

// U0 on the nonnegative octant of the twofold-padded frequency grid
// (Eq. (FUk), read with the unshifted basis), for the Coulomb kernel
// U(y) = 1/(4 pi |y|) on D_2L = prod [-2L_a, 2L_a] at nu_a = pi k_a / (2L_a),
// |k_a| = 0..N_a.  1/|y| = (2/sqrt(pi)) int_0^inf e^{-s^2 |y|^2} ds separates
// the box integral: U0 = (1/(2 pi^{3/2})) int_0^inf prod_a I_a(s) ds, the
// s-integral by the trapezoidal rule in tau = ln s with step 0.1 over
// [ln(1e-20 / prod_a 4 L_a), ln(pi^{3/2} 1e20) / 2], where the integrand is
// analytic in a strip and decays exponentially at both ends (the rule
// converges geometrically in 1/step).
void build_U0(Plan& P) {
  const double ht = 0.1;
  double a[3], prod2a = 1.0;
  for (int d = 0; d < 3; ++d) {
    a[d] = 2.0 * P.g.L[d];
    prod2a *= 2.0 * a[d];
  }
  const double tlo = std::log(1e-20 / prod2a);
  const double thi = 0.5 * std::log(std::pow(kPi, 1.5) * 1e20);
  const int nq = (int)std::ceil((thi - tlo) / ht) + 1;
  std::vector<double> s(nq), wq(nq);
  for (int q = 0; q < nq; ++q) {
    s[q] = std::exp(tlo + ht * q);
    wq[q] = ht * s[q];  // ds = s dtau
  }
  std::vector<double> T[3];
  for (int d = 0; d < 3; ++d) {
    const int Na = P.g.N[d];
    T[d].assign((size_t)(Na + 1) * nq, 0.0);
#pragma omp parallel for num_threads(P.threads) schedule(static)
    for (int k = 0; k <= Na; ++k)
      for (int q = 0; q < nq; ++q) T[d][(size_t)k * nq + q] = axis_integral(k, a[d], s[q]);
  }
  const int Nx = P.g.N[0], Ny = P.g.N[1], Nz = P.g.N[2];
  P.U0.assign((size_t)(Nx + 1) * (Ny + 1) * (Nz + 1), 0.0);
  const double c = 1.0 / (2.0 * std::pow(kPi, 1.5));
#pragma omp parallel for num_threads(P.threads) schedule(static)
  for (int kz = 0; kz <= Nz; ++kz)
    for (int ky = 0; ky <= Ny; ++ky)
      for (int kx = 0; kx <= Nx; ++kx) {
        const double* tx = &T[0][(size_t)kx * nq];
        const double* ty = &T[1][(size_t)ky * nq];
        const double* tz = &T[2][(size_t)kz * nq];
        double acc = 0.0;
        for (int q = 0; q < nq; ++q) acc += wq[q] * tx[q] * ty[q] * tz[q];
        P.U0[((size_t)kz * (Ny + 1) + ky) * (Nx + 1) + kx] = c * acc;
      }
}

// K(k) = -1 + 3 (n.nu_k)^2 U0(nu_k) on the full padded grid, from the
// Coulomb reformulation Phi = -rho - 3 U * (d_nn rho) (Eq. (DDI2Cou3D)); the
// spectral d_nn has the multiplier -(n.nu)^2.
void build_K(Plan& P) {
  const int Nx = P.g.N[0], Ny = P.g.N[1], Nz = P.g.N[2];
  const int Mx = 2 * Nx, My = 2 * Ny, Mz = 2 * Nz;
  P.K.assign((size_t)Mx * My * Mz, 0.0);
#pragma omp parallel for num_threads(P.threads) schedule(static)
  for (int mz = 0; mz < Mz; ++mz)
    for (int my = 0; my < My; ++my)
      for (int mx = 0; mx < Mx; ++mx) {
        const int kx = kfreq(mx, Mx), ky = kfreq(my, My), kz = kfreq(mz, Mz);
        const double nx = kPi * kx / (2.0 * P.g.L[0]), ny = kPi * ky / (2.0 * P.g.L[1]),
                     nz = kPi * kz / (2.0 * P.g.L[2]);
        const double nn = P.dip[0] * nx + P.dip[1] * ny + P.dip[2] * nz;
        const int ax = kx < 0 ? -kx : kx, ay = ky < 0 ? -ky : ky, az = kz < 0 ? -kz : kz;
        const double u0 = P.U0[((size_t)az * (Ny + 1) + ay) * (Nx + 1) + ax];
        P.K[((size_t)mz * My + my) * Mx + mx] = -1.0 + 3.0 * nn * nn * u0;
      }
}

// ---------------------------------------------------------------- sums
// sum over the grid of f(j), taken per z-plane in index order and then over
// the planes in order (independent of the thread count)
template <typename F> double grid_sum(const Plan& P, F f) {
  const long plane = (long)P.g.N[0] * P.g.N[1];
  const int Nz = P.g.N[2];
  std::vector<double> part(Nz, 0.0);
#pragma omp parallel for num_threads(P.threads) schedule(static)
  for (int z = 0; z < Nz; ++z) {
    double acc = 0.0;
    for (long j = z * plane; j < (z + 1) * plane; ++j) acc += f(j);
    part[z] = acc;
  }
  double s = 0.0;
  for (int z = 0; z < Nz; ++z) s += part[z];
  return s;
}

// <U, V> = Re(h_x h_y h_z sum_j U_j conj(V_j))  (Eq. (innerPro))
double inner(const Plan& P, const cx* U, const cx* V) {
  return P.g.hvol * grid_sum(P, [&](long j) { return U[j].re * V[j].re + U[j].im * V[j].im; });
}
double norm(const Plan& P, const cx* U) { return std::sqrt(inner(P, U, U)); }

using Vec = std::vector<cx>;

// ---------------------------------------------------------------- §2.2 ATKM
// Three-step apply: zero-pad rho to the twofold grid (indices [0, N) hold
// rho), FFT (Eq. (fouriercoeff)), multiply by K, inverse FFT (Eq.
// (U_TrunFour)), real part, crop to [0, N).
void atkm_apply(const Plan& P, const double* rho, double* out) {
  const int Nx = P.g.N[0], Ny = P.g.N[1], Nz = P.g.N[2];
  const int Mx = 2 * Nx, My = 2 * Ny, Mz = 2 * Nz;
  Vec pad((size_t)Mx * My * Mz, cx{0.0, 0.0});
#pragma omp parallel for num_threads(P.threads) schedule(static)
  for (int z = 0; z < Nz; ++z)
    for (int y = 0; y < Ny; ++y)
      for (int x = 0; x < Nx; ++x) pad[((size_t)z * My + y) * Mx + x] = {rho[((size_t)z * Ny + y) * Nx + x], 0.0};
  fft3(pad.data(), Mx, My, Mz, -1, *P.px, *P.py, *P.pz, P.threads);
#pragma omp parallel for num_threads(P.threads) schedule(static)
  for (long j = 0; j < (long)pad.size(); ++j) pad[j] = cscale(pad[j], P.K[j]);
  fft3(pad.data(), Mx, My, Mz, +1, *P.px, *P.py, *P.pz, P.threads);
#pragma omp parallel for num_threads(P.threads) schedule(static)
  for (int z = 0; z < Nz; ++z)
    for (int y = 0; y < Ny; ++y)
      for (int x = 0; x < Nx; ++x) out[((size_t)z * Ny + y) * Nx + x] = pad[((size_t)z * My + y) * Mx + x].re;
}

// ---------------------------------------------------------------- §2.1 operators
// sum_k mult_k fhat_k W_k at the grid points (Eq. (Fourphi)-(Laplacian));
// mult(kx, ky, kz) receives the frequencies nu of the index.
template <typename M> Vec spectral_apply(const Plan& P, const cx* f, M mult) {
  const int Nx = P.g.N[0], Ny = P.g.N[1], Nz = P.g.N[2];
  Vec a(f, f + P.g.n);
  fft3(a.data(), Nx, Ny, Nz, -1, *P.dx, *P.dy, *P.dz, P.threads);
#pragma omp parallel for num_threads(P.threads) schedule(static)
  for (int z = 0; z < Nz; ++z)
    for (int y = 0; y < Ny; ++y)
      for (int x = 0; x < Nx; ++x) {
        const size_t j = ((size_t)z * Ny + y) * Nx + x;
        a[j] = cmul(a[j], mult(P.nux[x], P.nuy[y], P.nuz[z]));
      }
  fft3(a.data(), Nx, Ny, Nz, +1, *P.dx, *P.dy, *P.dz, P.threads);
  return a;
}

// [[Delta]] f: multiplier -(nu_x^2 + nu_y^2 + nu_z^2)  (Eq. (Laplacian))
Vec laplacian(const Plan& P, const cx* f) {
  return spectral_apply(P, f, [](double a, double b, double c) { return cx{-(a * a + b * b + c * c), 0.0}; });
}
// [[d_x]] f, [[d_y]] f: multipliers i nu_x, i nu_y (Nyquist kept literally)
Vec d_dx(const Plan& P, const cx* f) {
  return spectral_apply(P, f, [](double a, double, double) { return cx{0.0, a}; });
}
Vec d_dy(const Plan& P, const cx* f) {
  return spectral_apply(P, f, [](double, double b, double) { return cx{0.0, b}; });
}
// [[L_z]] f = -i (x [[d_y]] f - y [[d_x]] f)  (Eq. (Laplacian))
Vec L_z(const Plan& P, const cx* f) {
  const Vec fy = d_dy(P, f), fx = d_dx(P, f);
  const int Nx = P.g.N[0], Ny = P.g.N[1], Nz = P.g.N[2];
  Vec o(P.g.n);
  for (int z = 0; z < Nz; ++z)
    for (int y = 0; y < Ny; ++y)
      for (int x = 0; x < Nx; ++x) {
        const size_t j = ((size_t)z * Ny + y) * Nx + x;
        const cx v = csub(cscale(fy[j], P.xc[x]), cscale(fx[j], P.yc[y]));
        o[j] = {v.im, -v.re};  // -i v
      }
  return o;
}
// V = (gamma_x^2 x^2 + gamma_y^2 y^2 + gamma_z^2 z^2) / 2  (Eq. (Vpoten))
double trap(const Plan& P, const double* gam, long j) {
  const int Nx = P.g.N[0], Ny = P.g.N[1];
  const int x = (int)(j % Nx), y = (int)((j / Nx) % Ny), z = (int)(j / ((long)Nx * Ny));
  return 0.5 * (gam[0] * gam[0] * P.xc[x] * P.xc[x] + gam[1] * gam[1] * P.yc[y] * P.yc[y] +
                gam[2] * gam[2] * P.zc[z] * P.zc[z]);
}

struct Phys {
  double gamma[3], beta, lam, Omega;
};

// H_phi f = -1/2 [[Delta]] f + V f + beta |phi|^2 f + lambda Phi f - Omega [[L_z]] f  (§2.3)
Vec apply_H(const Plan& P, const Phys& q, const cx* f, const cx* phi, const double* Phi) {
  const Vec lap = laplacian(P, f), lz = L_z(P, f);
  Vec o(P.g.n);
#pragma omp parallel for num_threads(P.threads) schedule(static)
  for (long j = 0; j < P.g.n; ++j) {
    const double V = trap(P, q.gamma, j);
    const double w = V + q.beta * (phi[j].re * phi[j].re + phi[j].im * phi[j].im) + q.lam * Phi[j];
    o[j] = csub(cadd(cscale(lap[j], -0.5), cscale(f[j], w)), cscale(lz[j], q.Omega));
  }
  return o;
}

// Terms of the discrete energy (§2.3) and the virial residual of Eq. (vir_iden).
struct Parts {
  double E_kin, E_pot, E_int, E_dip, E_rot, E, virial;
};
Parts energy_parts(const Plan& P, const Phys& q, const cx* phi, const double* Phi) {
  const long n = P.g.n;
  const Vec lap = laplacian(P, phi), lz = L_z(P, phi);
  Vec t(n);
  Parts e;
  for (long j = 0; j < n; ++j) t[j] = cscale(lap[j], -0.5);
  e.E_kin = inner(P, t.data(), phi);
  for (long j = 0; j < n; ++j) t[j] = cscale(phi[j], trap(P, q.gamma, j));
  e.E_pot = inner(P, t.data(), phi);
  for (long j = 0; j < n; ++j)
    t[j] = cscale(phi[j], 0.5 * q.beta * (phi[j].re * phi[j].re + phi[j].im * phi[j].im));
  e.E_int = inner(P, t.data(), phi);
  for (long j = 0; j < n; ++j) t[j] = cscale(phi[j], 0.5 * q.lam * Phi[j]);
  e.E_dip = inner(P, t.data(), phi);
  for (long j = 0; j < n; ++j) t[j] = cscale(lz[j], -q.Omega);
  e.E_rot = inner(P, t.data(), phi);
  e.E = e.E_kin + e.E_pot + e.E_int + e.E_dip + e.E_rot;
  e.virial = 2 * e.E_kin - 2 * e.E_pot + 3 * e.E_int + 3 * e.E_dip;
  return e;
}

// J_phi(f) = f - <f, phi> phi  (§2.3)
Vec project(const Plan& P, const cx* f, const cx* phi) {
  const double c = inner(P, f, phi);
  Vec o(P.g.n);
  for (long j = 0; j < P.g.n; ++j) o[j] = csub(f[j], cscale(phi[j], c));
  return o;
}

// alpha_Delta = alpha_V = <-1/2[[Delta]]phi + V phi + beta|phi|^2 phi, phi> + |lambda <Phi phi, phi>|  (§2.3)
double precond_shift(const Plan& P, const Phys& q, const cx* phi, const double* Phi) {
  const long n = P.g.n;
  const Vec lap = laplacian(P, phi);
  Vec t(n), u(n);
  for (long j = 0; j < n; ++j) {
    const double w = trap(P, q.gamma, j) + q.beta * (phi[j].re * phi[j].re + phi[j].im * phi[j].im);
    t[j] = cadd(cscale(lap[j], -0.5), cscale(phi[j], w));
    u[j] = cscale(phi[j], Phi[j]);
  }
  return inner(P, t.data(), phi) + std::fabs(q.lam * inner(P, u.data(), phi));
}

// P r = P_V^{1/2} P_Delta P_V^{1/2} r, P_Delta = (alpha - [[Delta]]/2)^{-1},
// P_V = (alpha + V + beta|phi|^2 + |lambda|(1 + sign Phi) Phi / 2)^{-1}  (§2.3)
Vec apply_precond(const Plan& P, const Phys& q, const cx* r, const cx* phi, const double* Phi, double alpha) {
  const long n = P.g.n;
  std::vector<double> sq(n);
  Vec t(n);
  for (long j = 0; j < n; ++j) {
    const double sg = Phi[j] > 0.0 ? 1.0 : (Phi[j] < 0.0 ? -1.0 : 0.0);
    const double pv = 1.0 / (alpha + trap(P, q.gamma, j) + q.beta * (phi[j].re * phi[j].re + phi[j].im * phi[j].im) +
                             std::fabs(q.lam) * (1.0 + sg) * Phi[j] / 2.0);
    sq[j] = std::sqrt(pv);
    t[j] = cscale(r[j], sq[j]);
  }
  Vec o = spectral_apply(P, t.data(), [alpha](double a, double b, double c) {
    return cx{1.0 / (alpha + 0.5 * (a * a + b * b + c * c)), 0.0};
  });
  for (long j = 0; j < n; ++j) o[j] = cscale(o[j], sq[j]);
  return o;
}

std::vector<double> density(const Plan& P, const cx* phi) {
  std::vector<double> rho(P.g.n);
  for (long j = 0; j < P.g.n; ++j) rho[j] = phi[j].re * phi[j].re + phi[j].im * phi[j].im;
  return rho;
}

std::vector<double> dipolar(const Plan& P, const std::vector<double>& rho) {
  std::vector<double> out(P.g.n);
  atkm_apply(P, rho.data(), out.data());
  return out;
}

double energy(const Plan& P, const Phys& q, const cx* phi, const double* Phi) { return energy_parts(P, q, phi, Phi).E; }

}  // namespace

// ================================================================== C ABI
extern "C" {

typedef struct ora_log {
  int n, halvings, reset, accepted, has_step, pad_;
  double E, mu, residual, linf_step, alpha, beta_cg, d1, curv, t0, t;
  double wall;  // seconds since the call began, when iteration n began (for timing only)
} ora_log;

typedef struct ora_result {
  double E, mu, E_kin, E_pot, E_int, E_dip, E_rot, virial, residual, linf_step;
  int iters, halvings, status, log_count;
} ora_result;

enum { ORA_OK = 0, ORA_NOT_CONVERGED = 5, ORA_STAGNATED = 6, ORA_ERR_NAN = 7, ORA_ERR_ARG = 1 };

// Number of OpenMP threads the library may use (1 when built without OpenMP).
int ora_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

// In-place 1D DFT of n interleaved complex values, y_k = sum_j x_j e^{sign 2 pi i jk/n} (unscaled).
int ora_dft1(double* data, int n, int sign) {
  if (n < 1 || !data) return ORA_ERR_ARG;
  Dft D(n);
  std::vector<cx> x(n), y(n);
  std::memcpy(x.data(), data, sizeof(cx) * n);
  D.apply(x.data(), y.data(), sign < 0 ? -1 : 1);
  std::memcpy(data, y.data(), sizeof(cx) * n);
  return ORA_OK;
}

// In-place 3D DFT of a [nz][ny][nx] complex array; sign -1 scaled by 1/(nx ny nz).
int ora_fft3(double* data, int nx, int ny, int nz, int sign, int threads) {
  if (!data || nx < 1 || ny < 1 || nz < 1) return ORA_ERR_ARG;
  Dft Dx(nx), Dy(ny), Dz(nz);
  fft3(reinterpret_cast<cx*>(data), nx, ny, nz, sign < 0 ? -1 : 1, Dx, Dy, Dz, threads < 1 ? 1 : threads);
  return ORA_OK;
}

// w(z) for count interleaved complex points z (Im z > 0).
int ora_faddeeva(const double* z, double* w, long count) {
  for (long i = 0; i < count; ++i) {
    const cx r = faddeeva(cx{z[2 * i], z[2 * i + 1]});
    w[2 * i] = r.re;
    w[2 * i + 1] = r.im;
  }
  return ORA_OK;
}

void* ora_plan_create(const int N[3], const double L[3], const double n[3], int threads) {
  for (int d = 0; d < 3; ++d)
    if (N[d] < 2 || N[d] % 2 || !(L[d] > 0.0)) return nullptr;
  const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  if (std::fabs(nn - 1.0) > 1e-12) return nullptr;
  Plan* P = new Plan();
  P->threads = threads < 1 ? 1 : threads;
  P->g.n = 1;
  P->g.hvol = 1.0;
  for (int d = 0; d < 3; ++d) {
    P->g.N[d] = N[d];
    P->g.L[d] = L[d];
    P->g.h[d] = 2.0 * L[d] / N[d];
    P->g.hvol *= P->g.h[d];
    P->g.n *= N[d];
    P->dip[d] = n[d];
  }
  std::vector<double>* xs[3] = {&P->xc, &P->yc, &P->zc};
  std::vector<double>* ns[3] = {&P->nux, &P->nuy, &P->nuz};
  for (int d = 0; d < 3; ++d) {
    xs[d]->resize(N[d]);
    ns[d]->resize(N[d]);
    for (int j = 0; j < N[d]; ++j) {
      (*xs[d])[j] = -L[d] + j * P->g.h[d];             // x_j = -L + j h  (§2.1)
      (*ns[d])[j] = kPi * kfreq(j, N[d]) / L[d];       // nu_k = pi k / L, FFT order
    }
  }
  P->dx = new Dft(N[0]);
  P->dy = new Dft(N[1]);
  P->dz = new Dft(N[2]);
  P->px = new Dft(2 * N[0]);
  P->py = new Dft(2 * N[1]);
  P->pz = new Dft(2 * N[2]);
  build_U0(*P);
  build_K(*P);
  return P;
}

void ora_plan_destroy(void* h) {
  Plan* P = static_cast<Plan*>(h);
  if (!P) return;
  delete P->dx; delete P->dy; delete P->dz; delete P->px; delete P->py; delete P->pz;
  delete P;
}

void ora_plan_set_threads(void* h, int threads) { static_cast<Plan*>(h)->threads = threads < 1 ? 1 : threads; }

void ora_plan_U0(void* h, double* out) {
  const Plan& P = *static_cast<Plan*>(h);
  std::memcpy(out, P.U0.data(), sizeof(double) * P.U0.size());
}

void ora_plan_K(void* h, double* out) {
  const Plan& P = *static_cast<Plan*>(h);
  std::memcpy(out, P.K.data(), sizeof(double) * P.K.size());
}

void ora_dipolar_potential(void* h, const double* rho, double* phi) {
  atkm_apply(*static_cast<Plan*>(h), rho, phi);
}

static Phys phys(const double* prm) {  // {gx, gy, gz, beta, lambda, Omega}
  Phys q;
  q.gamma[0] = prm[0]; q.gamma[1] = prm[1]; q.gamma[2] = prm[2];
  q.beta = prm[3]; q.lam = prm[4]; q.Omega = prm[5];
  return q;
}

void ora_apply_H(void* h, const double* prm, const double* f, const double* phi, const double* Phi, double* out) {
  const Plan& P = *static_cast<Plan*>(h);
  const Vec o = apply_H(P, phys(prm), reinterpret_cast<const cx*>(f), reinterpret_cast<const cx*>(phi), Phi);
  std::memcpy(out, o.data(), sizeof(cx) * P.g.n);
}

// out = {E_kin, E_pot, E_int, E_dip, E_rot, E, virial, mu}
void ora_energy_parts(void* h, const double* prm, const double* phi, const double* Phi, double* out) {
  const Plan& P = *static_cast<Plan*>(h);
  const Phys q = phys(prm);
  const cx* p = reinterpret_cast<const cx*>(phi);
  const Parts e = energy_parts(P, q, p, Phi);
  const Vec H = apply_H(P, q, p, p, Phi);
  const double vals[8] = {e.E_kin, e.E_pot, e.E_int, e.E_dip, e.E_rot, e.E, e.virial, inner(P, H.data(), p)};
  std::memcpy(out, vals, sizeof(vals));
}

double ora_inner(void* h, const double* u, const double* v) {
  return inner(*static_cast<Plan*>(h), reinterpret_cast<const cx*>(u), reinterpret_cast<const cx*>(v));
}

double ora_precond_shift(void* h, const double* prm, const double* phi, const double* Phi) {
  return precond_shift(*static_cast<Plan*>(h), phys(prm), reinterpret_cast<const cx*>(phi), Phi);
}

void ora_apply_precond(void* h, const double* prm, const double* r, const double* phi, const double* Phi,
                       double alpha, double* out) {
  const Plan& P = *static_cast<Plan*>(h);
  const Vec o = apply_precond(P, phys(prm), reinterpret_cast<const cx*>(r), reinterpret_cast<const cx*>(phi), Phi,
                              alpha);
  std::memcpy(out, o.data(), sizeof(cx) * P.g.n);
}

// Algorithm 1 (PCG-ATKM) with the step control of §2.3 (i)-(iii).
//   opts = {tol_residual, tol_linf, max_iter, max_halvings, energy_tol_ulps}
//   psi: N complex, initial data in, final state out.  Phi_out: N doubles (may be NULL).
int ora_pcg(void* h, const double* prm, const double* opts, double* psi, double* Phi_out, ora_result* res,
            ora_log* log, int log_cap) {
  const Plan& P = *static_cast<Plan*>(h);
  const Phys q = phys(prm);
  const double tol_res = opts[0], tol_linf = opts[1], tol_ulps = opts[4];
  const int max_iter = (int)opts[2], max_halv = (int)opts[3];
  const long n = P.g.n;
  const double eps = 2.220446049250313e-16;
  const auto start = std::chrono::steady_clock::now();
  Vec phi(reinterpret_cast<const cx*>(psi), reinterpret_cast<const cx*>(psi) + n);
  {
    const double nr = norm(P, phi.data());
    for (long j = 0; j < n; ++j) phi[j] = cscale(phi[j], 1.0 / nr);
  }
  std::vector<double> Phi = dipolar(P, density(P, phi.data()));  // Step 1 (n = 0)
  double E = energy(P, q, phi.data(), Phi.data());
  Vec p_prev, r_prev;
  double den_prev = 0.0;
  bool force_sd = false;
  int caps = 0, total_h = 0, status = ORA_NOT_CONVERGED, it = 0, logc = 0;
  double linf = INFINITY, mu = 0.0, res_norm = 0.0;
  while (true) {
    // Step 2: residual and chemical potential
    Vec Hphi = apply_H(P, q, phi.data(), phi.data(), Phi.data());
    mu = inner(P, Hphi.data(), phi.data());
    Vec r(n);
    for (long j = 0; j < n; ++j) r[j] = csub(Hphi[j], cscale(phi[j], mu));
    res_norm = norm(P, r.data());
    ora_log* L = (log && logc < log_cap) ? &log[logc++] : nullptr;
    if (L) {
      std::memset(L, 0, sizeof(*L));
      L->n = it; L->E = E; L->mu = mu; L->residual = res_norm; L->linf_step = linf;
      L->wall = std::chrono::duration<double>(std::chrono::steady_clock::now() - start).count();
    }
    if (!std::isfinite(E) || !std::isfinite(res_norm)) { status = ORA_ERR_NAN; break; }
    if (res_norm <= tol_res || (tol_linf > 0 && linf <= tol_linf)) { status = ORA_OK; break; }
    if (it >= max_iter) { status = ORA_NOT_CONVERGED; break; }
    // Step 3: preconditioned conjugate direction (Polak-Ribiere+)
    const double alpha = precond_shift(P, q, phi.data(), Phi.data());
    const Vec Pr = apply_precond(P, q, r.data(), phi.data(), Phi.data(), alpha);
    const Vec JPr = project(P, Pr.data(), phi.data());
    const double den = inner(P, r.data(), JPr.data());
    Vec mPr(n);
    for (long j = 0; j < n; ++j) mPr[j] = cscale(Pr[j], -1.0);
    const Vec d = project(P, mPr.data(), phi.data());
    double beta_cg = 0.0;
    Vec p;
    if (it > 0 && !force_sd) {
      const Vec Jr = project(P, r_prev.data(), phi.data());
      Vec dr(n);
      for (long j = 0; j < n; ++j) dr[j] = csub(r[j], Jr[j]);
      const double num = inner(P, dr.data(), JPr.data());
      beta_cg = num / den_prev > 0.0 ? num / den_prev : 0.0;
      const Vec Jp = project(P, p_prev.data(), phi.data());
      p.resize(n);
      for (long j = 0; j < n; ++j) p[j] = cadd(d[j], cscale(Jp[j], beta_cg));
    } else {
      p = d;
    }
    // Step 4 (i): fall back to preconditioned steepest descent if needed
    double d1 = inner(P, Hphi.data(), p.data());
    bool reset = false;
    if (d1 >= 0.0) {
      p = d;
      beta_cg = 0.0;
      reset = true;
      d1 = inner(P, Hphi.data(), p.data());
    }
    // Step 4 (ii): quadratic model of Q(t) = E(R_phi(t p)), Eq. (Energy_Expend)
    const Vec Hp = apply_H(P, q, p.data(), phi.data(), Phi.data());
    std::vector<double> rho1(n);
    for (long j = 0; j < n; ++j) rho1[j] = phi[j].re * p[j].re + phi[j].im * p[j].im;  // Re(conj(phi) p)
    const std::vector<double> Phi1 = dipolar(P, rho1);
    Vec gn(n);
    for (long j = 0; j < n; ++j) gn[j] = cscale(phi[j], 2.0 * (q.beta * rho1[j] + q.lam * Phi1[j]));
    const double pn2 = inner(P, p.data(), p.data());
    const double curv = inner(P, Hp.data(), p.data()) + inner(P, gn.data(), p.data()) - mu * pn2;
    double t = curv > 0.0 ? -d1 / curv : 0.3;
    const double t0 = t;
    const double pn = std::sqrt(pn2);
    // Step 4 (iii) + Step 5: retraction, halve until the energy decreases
    const double tolE = tol_ulps * eps * std::fabs(E);
    bool accepted = false, have_best = false;
    double bestE = 0.0, best_t = 0.0;
    Vec best_phi, phin(n);
    std::vector<double> best_Phi, Phin;
    double En = 0.0;
    int nh = 0;
    while (true) {
      const double c = std::cos(t * pn), s = std::sin(t * pn);
      for (long j = 0; j < n; ++j) phin[j] = cadd(cscale(phi[j], c), cscale(p[j], s / pn));
      const double nr = norm(P, phin.data());
      for (long j = 0; j < n; ++j) phin[j] = cscale(phin[j], 1.0 / nr);
      Phin = dipolar(P, density(P, phin.data()));
      En = energy(P, q, phin.data(), Phin.data());
      if (En <= E + tolE) { accepted = true; break; }
      if (!have_best || En < bestE) {
        have_best = true; bestE = En; best_phi = phin; best_Phi = Phin; best_t = t;
      }
      if (nh >= max_halv) break;
      t *= 0.5;
      ++nh;
    }
    total_h += nh;
    if (accepted) {
      caps = 0;
      force_sd = false;
    } else {
      En = bestE; phin = best_phi; Phin = best_Phi; t = best_t;
      ++caps;
      force_sd = true;
    }
    if (L) {
      L->alpha = alpha; L->beta_cg = beta_cg; L->reset = reset; L->d1 = d1; L->curv = curv; L->t0 = t0; L->t = t;
      L->halvings = nh; L->accepted = accepted; L->has_step = 1;
    }
    double m = 0.0;
    for (long j = 0; j < n; ++j) {
      const double dx = phin[j].re - phi[j].re, dy = phin[j].im - phi[j].im;
      const double a = std::sqrt(dx * dx + dy * dy);
      if (a > m) m = a;
    }
    linf = m;
    r_prev = r; p_prev = p; den_prev = den;
    phi = phin; Phi = Phin; E = En;
    ++it;
    if (caps >= 3) {
      status = ORA_STAGNATED;
      const Vec H2 = apply_H(P, q, phi.data(), phi.data(), Phi.data());
      mu = inner(P, H2.data(), phi.data());
      Vec r2(n);
      for (long j = 0; j < n; ++j) r2[j] = csub(H2[j], cscale(phi[j], mu));
      res_norm = norm(P, r2.data());
      break;
    }
  }
  const Parts e = energy_parts(P, q, phi.data(), Phi.data());
  std::memcpy(psi, phi.data(), sizeof(cx) * n);
  if (Phi_out) std::memcpy(Phi_out, Phi.data(), sizeof(double) * n);
  res->E = e.E; res->mu = mu; res->E_kin = e.E_kin; res->E_pot = e.E_pot; res->E_int = e.E_int;
  res->E_dip = e.E_dip; res->E_rot = e.E_rot; res->virial = e.virial; res->residual = res_norm;
  res->linf_step = linf; res->iters = it; res->halvings = total_h; res->status = status; res->log_count = logc;
  return status;
}

// Fourier interpolant (Eq. (Fourphi)) of a coarse grid function on a finer
// grid of the same box (Algorithm 2, Step 2): the coefficients of k in
// Lambda_Nc keep their k on the fine grid, every other coefficient is zero.
int ora_spectral_upsample(const int Nc[3], const double* psi_c, const int Nf[3], double* psi_f, int threads) {
  for (int d = 0; d < 3; ++d)
    if (Nf[d] < Nc[d]) return ORA_ERR_ARG;
  const long nc = (long)Nc[0] * Nc[1] * Nc[2], nf = (long)Nf[0] * Nf[1] * Nf[2];
  Vec c(reinterpret_cast<const cx*>(psi_c), reinterpret_cast<const cx*>(psi_c) + nc);
  Dft Cx(Nc[0]), Cy(Nc[1]), Cz(Nc[2]), Fx(Nf[0]), Fy(Nf[1]), Fz(Nf[2]);
  fft3(c.data(), Nc[0], Nc[1], Nc[2], -1, Cx, Cy, Cz, threads);
  Vec f(nf, cx{0.0, 0.0});
  for (int mz = 0; mz < Nc[2]; ++mz)
    for (int my = 0; my < Nc[1]; ++my)
      for (int mx = 0; mx < Nc[0]; ++mx) {
        const int kx = kfreq(mx, Nc[0]), ky = kfreq(my, Nc[1]), kz = kfreq(mz, Nc[2]);
        const long fx = (kx + Nf[0]) % Nf[0], fy = (ky + Nf[1]) % Nf[1], fz = (kz + Nf[2]) % Nf[2];
        f[(fz * Nf[1] + fy) * Nf[0] + fx] = c[((long)mz * Nc[1] + my) * Nc[0] + mx];
      }
  fft3(f.data(), Nf[0], Nf[1], Nf[2], +1, Fx, Fy, Fz, threads);
  std::memcpy(psi_f, f.data(), sizeof(cx) * nf);
  return ORA_OK;
}

}  // extern "C"
