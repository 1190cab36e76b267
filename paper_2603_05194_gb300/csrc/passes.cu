// Batched axis passes of the three spectral operators on the hot path:
//   * ATKM dipolar potential (§2.2): five passes on the twofold-padded grid,
//     x-forward (fused density formation and zero padding), y-forward,
//     z forward * K * inverse (fused multiplier), y-inverse, x-inverse (fused
//     real part and crop);
//   * H_phi f (§2.3 with the spectral operators of Eq. (Laplacian)): one
//     forward/multiply/inverse pass per axis, the x and y passes carrying the
//     rotation term -Omega L_z = i Omega (x d_y - y d_x), the z pass adding the
//     pointwise potential, with fused Parseval sums of the energy terms;
//   * the preconditioner P_V^{1/2} P_Delta P_V^{1/2} (§2.3): five passes with
//     P_V^{1/2} fused into the first and last.
// Every pass keeps whole lines in shared memory (FFT engine in
// atkm_internal.cuh); strided axes move T adjacent columns per CTA so global
// accesses stay coalesced.  R is the arithmetic/workspace type (double or
// float); the caller-visible vectors are always FP64.
#include "atkm_internal.cuh"

namespace atkm {

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

__device__ __forceinline__ int kfreq(int m, int M) { return m < (M >> 1) ? m : m - M; }

template <typename R> __device__ __forceinline__ cx<R> from64(double2 z) { return mk<R>((R)z.x, (R)z.y); }
template <typename R> __device__ __forceinline__ double2 to64(cx<R> z) { return make_double2((double)z.x, (double)z.y); }

template <typename R> __device__ __forceinline__ cx<R>* tile_ptr() {
  extern __shared__ __align__(16) unsigned char atkm_smem[];
  return reinterpret_cast<cx<R>*>(atkm_smem);
}

// ---------------------------------------------------------------- ATKM
template <typename R, int MODE>
__global__ void __launch_bounds__(kThreads)
k_atkm_x_fwd(const double* __restrict__ a, const double* __restrict__ b, cx<R>* __restrict__ W1,
             Geo g, FftLen f, int T) {
  cx<R>* tile = tile_ptr<R>();
  cx<R>* tw = tile + T * f.L;
  const int L = f.L;
  const long nlines = (long)g.Nz * g.Ny;
  const long line0 = (long)blockIdx.x * T;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int t = e / L, j = e - t * L;
    const long line = line0 + t;
    double v = 0.0;
    if (j < g.Nx && line < nlines) {
      const size_t idx = (size_t)line * g.Nx + j;
      if (MODE == SRC_RHO) {
        v = a[idx];
      } else if (MODE == SRC_PSI) {
        const double2 z = reinterpret_cast<const double2*>(a)[idx];
        v = z.x * z.x + z.y * z.y;
      } else {
        const double2 u = reinterpret_cast<const double2*>(a)[idx];
        const double2 w = reinterpret_cast<const double2*>(b)[idx];
        v = u.x * w.x + u.y * w.y;
      }
    }
    tile[e] = mk<R>((R)v, (R)0);
  }
  load_tw<R>(tw, f);
  __syncthreads();
  fft_tile<R, -1, true>(tile, tw, f, T);
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int t = e / L;
    const long line = line0 + t;
    if (line < nlines) W1[(size_t)line * L + (e - t * L)] = tile[e];
  }
}

// y forward: lines (z < Nz, kx < Mx), input rows y < Ny of W1, zero beyond.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_atkm_y_fwd(const cx<R>* __restrict__ W1, cx<R>* __restrict__ W2, Geo g, FftLen f, int T) {
  cx<R>* tile = tile_ptr<R>();
  cx<R>* tw = tile + T * f.L;
  const int L = f.L, z = blockIdx.y, x0 = blockIdx.x * T;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    cx<R> v = mk<R>((R)0, (R)0);
    if (j < g.Ny && x < g.Mx) v = W1[((size_t)z * g.Ny + j) * g.Mx + x];
    tile[e] = v;
  }
  load_tw<R>(tw, f);
  __syncthreads();
  fft_tile<R, -1, false>(tile, tw, f, T);
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    if (x < g.Mx) W2[((size_t)z * g.My + j) * g.Mx + x] = tile[e];
  }
}

// z: forward, times K(k)/(Mx My Mz), inverse, crop to z < Nz (in place).
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_atkm_z(cx<R>* __restrict__ W2, const double* __restrict__ U0, Geo g, FftLen f, int T,
         double n0, double n1, double n2, double invM) {
  cx<R>* tile = tile_ptr<R>();
  cx<R>* tw = tile + T * f.L;
  const int L = f.L, y = blockIdx.y, x0 = blockIdx.x * T;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    cx<R> v = mk<R>((R)0, (R)0);
    if (j < g.Nz && x < g.Mx) v = W2[((size_t)j * g.My + y) * g.Mx + x];
    tile[e] = v;
  }
  load_tw<R>(tw, f);
  __syncthreads();
  fft_tile<R, -1, false>(tile, tw, f, T);
  const int ky = kfreq(y, g.My);
  const double nuy = kPi * ky / (2.0 * g.Ly);
  const int aky = ky < 0 ? -ky : ky;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    if (x < g.Mx) {
      const int kx = kfreq(x, g.Mx), kz = kfreq(j, g.Mz);
      const int akx = kx < 0 ? -kx : kx, akz = kz < 0 ? -kz : kz;
      const double nux = kPi * kx / (2.0 * g.Lx), nuz = kPi * kz / (2.0 * g.Lz);
      const double nd = n0 * nux + n1 * nuy + n2 * nuz;
      const double u = U0[((size_t)akz * (g.Ny + 1) + aky) * (g.Nx + 1) + akx];
      const R K = (R)((-1.0 + 3.0 * nd * nd * u) * invM);
      tile[e] = scl<R>(tile[e], K);
    }
  }
  __syncthreads();
  fft_tile<R, 1, false>(tile, tw, f, T);
  for (int e = threadIdx.x; e < T * g.Nz; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    if (x < g.Mx) W2[((size_t)j * g.My + y) * g.Mx + x] = tile[e];
  }
}

// y inverse: lines (z < Nz, kx), output rows y < Ny into W1.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_atkm_y_inv(const cx<R>* __restrict__ W2, cx<R>* __restrict__ W1, Geo g, FftLen f, int T) {
  cx<R>* tile = tile_ptr<R>();
  cx<R>* tw = tile + T * f.L;
  const int L = f.L, z = blockIdx.y, x0 = blockIdx.x * T;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    cx<R> v = mk<R>((R)0, (R)0);
    if (x < g.Mx) v = W2[((size_t)z * g.My + j) * g.Mx + x];
    tile[e] = v;
  }
  load_tw<R>(tw, f);
  __syncthreads();
  fft_tile<R, 1, false>(tile, tw, f, T);
  for (int e = threadIdx.x; e < T * g.Ny; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    if (x < g.Mx) W1[((size_t)z * g.Ny + j) * g.Mx + x] = tile[e];
  }
}

// x inverse: lines (z, y), Phi = Re(.) for x < Nx.
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_atkm_x_inv(const cx<R>* __restrict__ W1, double* __restrict__ phi, Geo g, FftLen f, int T) {
  cx<R>* tile = tile_ptr<R>();
  cx<R>* tw = tile + T * f.L;
  const int L = f.L;
  const long nlines = (long)g.Nz * g.Ny;
  const long line0 = (long)blockIdx.x * T;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int t = e / L;
    const long line = line0 + t;
    cx<R> v = mk<R>((R)0, (R)0);
    if (line < nlines) v = W1[(size_t)line * L + (e - t * L)];
    tile[e] = v;
  }
  load_tw<R>(tw, f);
  __syncthreads();
  fft_tile<R, 1, true>(tile, tw, f, T);
  for (int e = threadIdx.x; e < T * g.Nx; e += kThreads) {
    const int t = e / g.Nx, j = e - t * g.Nx;
    const long line = line0 + t;
    if (line < nlines) phi[(size_t)line * g.Nx + j] = (double)tile[t * L + j].x;
  }
}

// ------------------------------------------------------------------ H f
// x pass: multiplier (nu^2/2 + Omega y nu)/Nx on lines (z, y).
template <typename R, bool RED>
__global__ void __launch_bounds__(kThreads)
k_H_x(const double2* __restrict__ fin, cx<R>* __restrict__ acc, Geo g, FftLen f, int T, double Omega,
      double* __restrict__ part, int pstride) {
  cx<R>* tile = tile_ptr<R>();
  cx<R>* tw = tile + T * f.L;
  const int L = f.L;  // Nx
  const long nlines = (long)g.Nz * g.Ny;
  const long line0 = (long)blockIdx.x * T;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int t = e / L;
    const long line = line0 + t;
    cx<R> v = mk<R>((R)0, (R)0);
    if (line < nlines) v = from64<R>(fin[(size_t)line * L + (e - t * L)]);
    tile[e] = v;
  }
  load_tw<R>(tw, f);
  __syncthreads();
  fft_tile<R, -1, true>(tile, tw, f, T);
  double s[2] = {0.0, 0.0};
  const double invL = 1.0 / L;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int t = e / L, j = e - t * L;
    const long line = line0 + t;
    const double y = -g.Ly + (double)(line % g.Ny) * g.hy;
    const double nu = kPi * kfreq(j, L) / g.Lx;
    const double mk_kin = 0.5 * nu * nu, mk_rot = Omega * y * nu;
    cx<R> c = tile[e];
    if (RED && line < nlines) {
      const double a2 = (double)c.x * c.x + (double)c.y * c.y;
      s[0] += mk_kin * a2 * invL;
      s[1] += mk_rot * a2 * invL;
    }
    tile[e] = scl<R>(c, (R)((mk_kin + mk_rot) * invL));
  }
  __syncthreads();
  fft_tile<R, 1, true>(tile, tw, f, T);
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int t = e / L;
    const long line = line0 + t;
    if (line < nlines) acc[(size_t)line * L + (e - t * L)] = tile[e];
  }
  if (RED) block_reduce_store<2>(s, part, pstride, blockIdx.x);
}

// y pass: multiplier (nu^2/2 - Omega x nu)/Ny on lines (z, x); acc += result.
template <typename R, bool RED>
__global__ void __launch_bounds__(kThreads)
k_H_y(const double2* __restrict__ fin, cx<R>* __restrict__ acc, Geo g, FftLen f, int T, double Omega,
      double* __restrict__ part, int pstride) {
  cx<R>* tile = tile_ptr<R>();
  cx<R>* tw = tile + T * f.L;
  const int L = f.L, z = blockIdx.y, x0 = blockIdx.x * T;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    cx<R> v = mk<R>((R)0, (R)0);
    if (x < g.Nx) v = from64<R>(fin[((size_t)z * g.Ny + j) * g.Nx + x]);
    tile[e] = v;
  }
  load_tw<R>(tw, f);
  __syncthreads();
  fft_tile<R, -1, false>(tile, tw, f, T);
  double s[2] = {0.0, 0.0};
  const double invL = 1.0 / L;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    const double xc = -g.Lx + (double)x * g.hx;
    const double nu = kPi * kfreq(j, L) / g.Ly;
    const double mk_kin = 0.5 * nu * nu, mk_rot = -Omega * xc * nu;
    cx<R> c = tile[e];
    if (RED && x < g.Nx) {
      const double a2 = (double)c.x * c.x + (double)c.y * c.y;
      s[0] += mk_kin * a2 * invL;
      s[1] += mk_rot * a2 * invL;
    }
    tile[e] = scl<R>(c, (R)((mk_kin + mk_rot) * invL));
  }
  __syncthreads();
  fft_tile<R, 1, false>(tile, tw, f, T);
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    if (x < g.Nx) {
      const size_t idx = ((size_t)z * g.Ny + j) * g.Nx + x;
      acc[idx] = add<R>(acc[idx], tile[e]);
    }
  }
  if (RED) block_reduce_store<2>(s, part, pstride, blockIdx.y * gridDim.x + blockIdx.x);
}

// z pass: multiplier nu^2/(2 Nz) on lines (y, x), then
// Hf = acc + result + (V + beta|phi|^2 + lambda Phi) f.
template <typename R, bool RED>
__global__ void __launch_bounds__(kThreads)
k_H_z(const double2* __restrict__ fin, const double2* __restrict__ phi, const double* __restrict__ Phi,
      const cx<R>* __restrict__ acc, double2* __restrict__ Hf, Geo g, FftLen f, int T, Phys ph,
      double* __restrict__ part, int pstride) {
  cx<R>* tile = tile_ptr<R>();
  cx<R>* tw = tile + T * f.L;
  const int L = f.L, y = blockIdx.y, x0 = blockIdx.x * T;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    cx<R> v = mk<R>((R)0, (R)0);
    if (x < g.Nx) v = from64<R>(fin[((size_t)j * g.Ny + y) * g.Nx + x]);
    tile[e] = v;
  }
  load_tw<R>(tw, f);
  __syncthreads();
  fft_tile<R, -1, false>(tile, tw, f, T);
  double s[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  const double invL = 1.0 / L;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    const double nu = kPi * kfreq(j, L) / g.Lz;
    const double m = 0.5 * nu * nu;
    cx<R> c = tile[e];
    if (RED && x < g.Nx) s[0] += m * ((double)c.x * c.x + (double)c.y * c.y) * invL;
    tile[e] = scl<R>(c, (R)(m * invL));
  }
  __syncthreads();
  fft_tile<R, 1, false>(tile, tw, f, T);
  const double yc = -g.Ly + (double)y * g.hy;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    if (x < g.Nx) {
      const size_t idx = ((size_t)j * g.Ny + y) * g.Nx + x;
      const double xc = -g.Lx + (double)x * g.hx, zc = -g.Lz + (double)j * g.hz;
      const double V = 0.5 * (ph.gx2 * xc * xc + ph.gy2 * yc * yc + ph.gz2 * zc * zc);
      const double2 fv = fin[idx], pv = phi[idx];
      const double rho = pv.x * pv.x + pv.y * pv.y;
      const double Pd = Phi[idx];
      const double w = V + ph.beta * rho + ph.lambda * Pd;
      const cx<R> kin = add<R>(acc[idx], tile[e]);
      double2 o;
      o.x = (double)kin.x + w * fv.x;
      o.y = (double)kin.y + w * fv.y;
      Hf[idx] = o;
      if (RED) {
        const double f2 = fv.x * fv.x + fv.y * fv.y;
        s[1] += V * f2;
        s[2] += f2 * f2;
        s[3] += Pd * f2;
        s[4] += o.x * fv.x + o.y * fv.y;
        s[5] += f2;
      }
    }
  }
  if (RED) block_reduce_store<6>(s, part, pstride, blockIdx.y * gridDim.x + blockIdx.x);
}

// ----------------------------------------------------------- preconditioner
__device__ __forceinline__ double pv_sqrt(const Geo& g, const Phys& ph, double alpha, int x, int y, int z,
                                          double2 pv, double Pd) {
  const double xc = -g.Lx + (double)x * g.hx, yc = -g.Ly + (double)y * g.hy, zc = -g.Lz + (double)z * g.hz;
  const double V = 0.5 * (ph.gx2 * xc * xc + ph.gy2 * yc * yc + ph.gz2 * zc * zc);
  const double den = alpha + V + ph.beta * (pv.x * pv.x + pv.y * pv.y) + fabs(ph.lambda) * fmax(Pd, 0.0);
  return 1.0 / sqrt(den);
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_P_x_fwd(const double2* __restrict__ r, const double2* __restrict__ phi, const double* __restrict__ Phi,
          cx<R>* __restrict__ Wk, Geo g, FftLen f, int T, Phys ph, const double* __restrict__ alpha_p) {
  cx<R>* tile = tile_ptr<R>();
  cx<R>* tw = tile + T * f.L;
  const int L = f.L;
  const long nlines = (long)g.Nz * g.Ny;
  const long line0 = (long)blockIdx.x * T;
  const double alpha = *alpha_p;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int t = e / L, j = e - t * L;
    const long line = line0 + t;
    cx<R> v = mk<R>((R)0, (R)0);
    if (line < nlines) {
      const size_t idx = (size_t)line * L + j;
      const double w = pv_sqrt(g, ph, alpha, j, (int)(line % g.Ny), (int)(line / g.Ny), phi[idx], Phi[idx]);
      const double2 rv = r[idx];
      v = mk<R>((R)(w * rv.x), (R)(w * rv.y));
    }
    tile[e] = v;
  }
  load_tw<R>(tw, f);
  __syncthreads();
  fft_tile<R, -1, true>(tile, tw, f, T);
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int t = e / L;
    const long line = line0 + t;
    if (line < nlines) Wk[(size_t)line * L + (e - t * L)] = tile[e];
  }
}

// Column transform of Wk along y (in place): lines (z, x).
template <typename R, int S>
__global__ void __launch_bounds__(kThreads)
k_col_y(cx<R>* __restrict__ Wk, Geo g, FftLen f, int T) {
  cx<R>* tile = tile_ptr<R>();
  cx<R>* tw = tile + T * f.L;
  const int L = f.L, z = blockIdx.y, x0 = blockIdx.x * T;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    cx<R> v = mk<R>((R)0, (R)0);
    if (x < g.Nx) v = Wk[((size_t)z * g.Ny + j) * g.Nx + x];
    tile[e] = v;
  }
  load_tw<R>(tw, f);
  __syncthreads();
  fft_tile<R, S, false>(tile, tw, f, T);
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    if (x < g.Nx) Wk[((size_t)z * g.Ny + j) * g.Nx + x] = tile[e];
  }
}

// z: forward, times 1/((alpha + |nu|^2/2) N), inverse (in place).
template <typename R>
__global__ void __launch_bounds__(kThreads)
k_P_z(cx<R>* __restrict__ Wk, Geo g, FftLen f, int T, const double* __restrict__ alpha_p) {
  cx<R>* tile = tile_ptr<R>();
  cx<R>* tw = tile + T * f.L;
  const int L = f.L, y = blockIdx.y, x0 = blockIdx.x * T;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    cx<R> v = mk<R>((R)0, (R)0);
    if (x < g.Nx) v = Wk[((size_t)j * g.Ny + y) * g.Nx + x];
    tile[e] = v;
  }
  load_tw<R>(tw, f);
  __syncthreads();
  fft_tile<R, -1, false>(tile, tw, f, T);
  const double alpha = *alpha_p;
  const double invN = 1.0 / ((double)g.Nx * g.Ny * g.Nz);
  const double nuy = kPi * kfreq(y, g.Ny) / g.Ly;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    const double nux = kPi * kfreq(x < g.Nx ? x : 0, g.Nx) / g.Lx;
    const double nuz = kPi * kfreq(j, L) / g.Lz;
    const double m = invN / (alpha + 0.5 * (nux * nux + nuy * nuy + nuz * nuz));
    tile[e] = scl<R>(tile[e], (R)m);
  }
  __syncthreads();
  fft_tile<R, 1, false>(tile, tw, f, T);
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int j = e / T, t = e - j * T, x = x0 + t;
    if (x < g.Nx) Wk[((size_t)j * g.Ny + y) * g.Nx + x] = tile[e];
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
k_P_x_inv(const cx<R>* __restrict__ Wk, const double2* __restrict__ phi, const double* __restrict__ Phi,
          double2* __restrict__ Pr, Geo g, FftLen f, int T, Phys ph, const double* __restrict__ alpha_p) {
  cx<R>* tile = tile_ptr<R>();
  cx<R>* tw = tile + T * f.L;
  const int L = f.L;
  const long nlines = (long)g.Nz * g.Ny;
  const long line0 = (long)blockIdx.x * T;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int t = e / L;
    const long line = line0 + t;
    cx<R> v = mk<R>((R)0, (R)0);
    if (line < nlines) v = Wk[(size_t)line * L + (e - t * L)];
    tile[e] = v;
  }
  load_tw<R>(tw, f);
  __syncthreads();
  fft_tile<R, 1, true>(tile, tw, f, T);
  const double alpha = *alpha_p;
  for (int e = threadIdx.x; e < T * L; e += kThreads) {
    const int t = e / L, j = e - t * L;
    const long line = line0 + t;
    if (line < nlines) {
      const size_t idx = (size_t)line * L + j;
      const double w = pv_sqrt(g, ph, alpha, j, (int)(line % g.Ny), (int)(line / g.Ny), phi[idx], Phi[idx]);
      const cx<R> c = tile[e];
      Pr[idx] = make_double2(w * (double)c.x, w * (double)c.y);
    }
  }
}

// Full padded multiplier in FFT order (test/inspection path).
__global__ void k_multiplier_full(double* __restrict__ K, const double* __restrict__ U0, Geo g, double n0,
                                  double n1, double n2) {
  const size_t total = (size_t)g.Mx * g.My * g.Mz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % g.Mx);
    const int y = (int)((i / g.Mx) % g.My);
    const int z = (int)(i / ((size_t)g.Mx * g.My));
    const int kx = kfreq(x, g.Mx), ky = kfreq(y, g.My), kz = kfreq(z, g.Mz);
    const double nd = n0 * kPi * kx / (2.0 * g.Lx) + n1 * kPi * ky / (2.0 * g.Ly) + n2 * kPi * kz / (2.0 * g.Lz);
    const double u = U0[((size_t)abs(kz) * (g.Ny + 1) + abs(ky)) * (g.Nx + 1) + abs(kx)];
    K[i] = -1.0 + 3.0 * nd * nd * u;
  }
}

// ------------------------------------------------------------ host helpers
inline int ceil_div(long a, long b) { return (int)((a + b - 1) / b); }

// Lines per CTA for line-major (x) passes: fill the tile, but keep at least
// two CTAs per SM on small grids.
template <typename R> int lm_tile(int L, long nlines) {
  int T = TileElems<R>::value / L;
  if (T < 1) T = 1;
  while (T > 1 && ceil_div(nlines, T) < 2 * 152) T >>= 1;
  return T;
}
// Columns per CTA for strided passes over X columns and `outer` tiles.
template <typename R> int col_tile(int L, int X, long outer) {
  int T = TileElems<R>::value / L;
  if (T > X) T = X;
  if (T < 1) T = 1;
  while (T > 8 && (long)ceil_div(X, T) * outer < 2 * 152) T >>= 1;
  return T;
}

template <typename R> size_t smem_bytes(int T, int L) { return (size_t)(T * L + L) * sizeof(cx<R>); }

template <typename K>
cudaError_t prep(K kernel) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)((kMaxElems + kMaxLen) * sizeof(double2)));
}

template <typename R> cx<R>* ws1(atkm_plan* p);
template <> double2* ws1<double>(atkm_plan* p) { return p->W1; }
template <> float2* ws1<float>(atkm_plan* p) { return p->W1f; }
template <typename R> cx<R>* ws2(atkm_plan* p);
template <> double2* ws2<double>(atkm_plan* p) { return p->W2; }
template <> float2* ws2<float>(atkm_plan* p) { return p->W2f; }
template <typename R> cx<R>* ws3(atkm_plan* p);
template <> double2* ws3<double>(atkm_plan* p) { return p->T1; }
template <> float2* ws3<float>(atkm_plan* p) { return p->T1f; }

}  // namespace

template <typename R>
cudaError_t launch_atkm(atkm_plan* p, int mode, const double* a, const double* b, double* phi, cudaStream_t st) {
  static bool prepared = false;
  if (!prepared) {
    cudaError_t e;
    if ((e = prep(k_atkm_x_fwd<R, SRC_RHO>)) != cudaSuccess) return e;
    if ((e = prep(k_atkm_x_fwd<R, SRC_PSI>)) != cudaSuccess) return e;
    if ((e = prep(k_atkm_x_fwd<R, SRC_PAIR>)) != cudaSuccess) return e;
    if ((e = prep(k_atkm_y_fwd<R>)) != cudaSuccess) return e;
    if ((e = prep(k_atkm_z<R>)) != cudaSuccess) return e;
    if ((e = prep(k_atkm_y_inv<R>)) != cudaSuccess) return e;
    if ((e = prep(k_atkm_x_inv<R>)) != cudaSuccess) return e;
    prepared = true;
  }
  const Geo& g = p->g;
  cx<R>* W1 = ws1<R>(p);
  cx<R>* W2 = ws2<R>(p);
  if (!W1 || !W2) return cudaErrorInvalidValue;
  const long nl = (long)g.Nz * g.Ny;
  const int Tx = lm_tile<R>(g.Mx, nl);
  const dim3 gx(ceil_div(nl, Tx));
  const size_t sx = smem_bytes<R>(Tx, g.Mx);
  if (mode == SRC_RHO) k_atkm_x_fwd<R, SRC_RHO><<<gx, kThreads, sx, st>>>(a, b, W1, g, p->fM[0], Tx);
  else if (mode == SRC_PSI) k_atkm_x_fwd<R, SRC_PSI><<<gx, kThreads, sx, st>>>(a, b, W1, g, p->fM[0], Tx);
  else k_atkm_x_fwd<R, SRC_PAIR><<<gx, kThreads, sx, st>>>(a, b, W1, g, p->fM[0], Tx);
  const int Ty = col_tile<R>(g.My, g.Mx, g.Nz);
  const dim3 gy(ceil_div(g.Mx, Ty), g.Nz);
  k_atkm_y_fwd<R><<<gy, kThreads, smem_bytes<R>(Ty, g.My), st>>>(W1, W2, g, p->fM[1], Ty);
  const int Tz = col_tile<R>(g.Mz, g.Mx, g.My);
  const dim3 gz(ceil_div(g.Mx, Tz), g.My);
  const double invM = 1.0 / ((double)g.Mx * g.My * g.Mz);
  k_atkm_z<R><<<gz, kThreads, smem_bytes<R>(Tz, g.Mz), st>>>(W2, p->U0, g, p->fM[2], Tz, p->n[0], p->n[1],
                                                              p->n[2], invM);
  k_atkm_y_inv<R><<<gy, kThreads, smem_bytes<R>(Ty, g.My), st>>>(W2, W1, g, p->fM[1], Ty);
  k_atkm_x_inv<R><<<gx, kThreads, sx, st>>>(W1, phi, g, p->fM[0], Tx);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_H(atkm_plan* p, const Phys& ph, const double* f, const double* phi, const double* Phi,
                     double* Hf, int red_slot, cudaStream_t st) {
  static bool prepared = false;
  if (!prepared) {
    cudaError_t e;
    if ((e = prep(k_H_x<R, true>)) != cudaSuccess) return e;
    if ((e = prep(k_H_x<R, false>)) != cudaSuccess) return e;
    if ((e = prep(k_H_y<R, true>)) != cudaSuccess) return e;
    if ((e = prep(k_H_y<R, false>)) != cudaSuccess) return e;
    if ((e = prep(k_H_z<R, true>)) != cudaSuccess) return e;
    if ((e = prep(k_H_z<R, false>)) != cudaSuccess) return e;
    prepared = true;
  }
  const Geo& g = p->g;
  cx<R>* acc = ws3<R>(p);
  if (!acc) return cudaErrorInvalidValue;
  const bool red = red_slot >= 0;
  const double2* fin = reinterpret_cast<const double2*>(f);
  const double2* pin = reinterpret_cast<const double2*>(phi);
  double2* out = reinterpret_cast<double2*>(Hf);
  cudaError_t e;
  // x
  const long nl = (long)g.Nz * g.Ny;
  const int Tx = lm_tile<R>(g.Nx, nl);
  const int bx = ceil_div(nl, Tx);
  if (red) k_H_x<R, true><<<bx, kThreads, smem_bytes<R>(Tx, g.Nx), st>>>(fin, acc, g, p->fN[0], Tx, ph.Omega, p->partials, bx);
  else k_H_x<R, false><<<bx, kThreads, smem_bytes<R>(Tx, g.Nx), st>>>(fin, acc, g, p->fN[0], Tx, ph.Omega, nullptr, 0);
  if (red && (e = launch_finalize(p, 2, bx, red_slot + 0, st)) != cudaSuccess) return e;
  // y
  const int Ty = col_tile<R>(g.Ny, g.Nx, g.Nz);
  const dim3 gy(ceil_div(g.Nx, Ty), g.Nz);
  const int by = gy.x * gy.y;
  if (red) k_H_y<R, true><<<gy, kThreads, smem_bytes<R>(Ty, g.Ny), st>>>(fin, acc, g, p->fN[1], Ty, ph.Omega, p->partials, by);
  else k_H_y<R, false><<<gy, kThreads, smem_bytes<R>(Ty, g.Ny), st>>>(fin, acc, g, p->fN[1], Ty, ph.Omega, nullptr, 0);
  if (red && (e = launch_finalize(p, 2, by, red_slot + 2, st)) != cudaSuccess) return e;
  // z
  const int Tz = col_tile<R>(g.Nz, g.Nx, g.Ny);
  const dim3 gz(ceil_div(g.Nx, Tz), g.Ny);
  const int bz = gz.x * gz.y;
  if (red) k_H_z<R, true><<<gz, kThreads, smem_bytes<R>(Tz, g.Nz), st>>>(fin, pin, Phi, acc, out, g, p->fN[2], Tz, ph, p->partials, bz);
  else k_H_z<R, false><<<gz, kThreads, smem_bytes<R>(Tz, g.Nz), st>>>(fin, pin, Phi, acc, out, g, p->fN[2], Tz, ph, nullptr, 0);
  if (red && (e = launch_finalize(p, 6, bz, red_slot + 4, st)) != cudaSuccess) return e;
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_precond(atkm_plan* p, const Phys& ph, const double* alpha_dev, const double* r,
                           const double* phi, const double* Phi, double* Pr, cudaStream_t st) {
  static bool prepared = false;
  if (!prepared) {
    cudaError_t e;
    if ((e = prep(k_P_x_fwd<R>)) != cudaSuccess) return e;
    if ((e = prep(k_col_y<R, -1>)) != cudaSuccess) return e;
    if ((e = prep(k_col_y<R, 1>)) != cudaSuccess) return e;
    if ((e = prep(k_P_z<R>)) != cudaSuccess) return e;
    if ((e = prep(k_P_x_inv<R>)) != cudaSuccess) return e;
    prepared = true;
  }
  const Geo& g = p->g;
  cx<R>* Wk = ws3<R>(p);
  if (!Wk) return cudaErrorInvalidValue;
  const double2* rin = reinterpret_cast<const double2*>(r);
  const double2* pin = reinterpret_cast<const double2*>(phi);
  double2* out = reinterpret_cast<double2*>(Pr);
  const long nl = (long)g.Nz * g.Ny;
  const int Tx = lm_tile<R>(g.Nx, nl);
  const int bx = ceil_div(nl, Tx);
  const size_t sx = smem_bytes<R>(Tx, g.Nx);
  k_P_x_fwd<R><<<bx, kThreads, sx, st>>>(rin, pin, Phi, Wk, g, p->fN[0], Tx, ph, alpha_dev);
  const int Ty = col_tile<R>(g.Ny, g.Nx, g.Nz);
  const dim3 gy(ceil_div(g.Nx, Ty), g.Nz);
  k_col_y<R, -1><<<gy, kThreads, smem_bytes<R>(Ty, g.Ny), st>>>(Wk, g, p->fN[1], Ty);
  const int Tz = col_tile<R>(g.Nz, g.Nx, g.Ny);
  const dim3 gz(ceil_div(g.Nx, Tz), g.Ny);
  k_P_z<R><<<gz, kThreads, smem_bytes<R>(Tz, g.Nz), st>>>(Wk, g, p->fN[2], Tz, alpha_dev);
  k_col_y<R, 1><<<gy, kThreads, smem_bytes<R>(Ty, g.Ny), st>>>(Wk, g, p->fN[1], Ty);
  k_P_x_inv<R><<<bx, kThreads, sx, st>>>(Wk, pin, Phi, out, g, p->fN[0], Tx, ph, alpha_dev);
  return cudaGetLastError();
}

cudaError_t launch_multiplier_full(const atkm_plan* p, double* dst, cudaStream_t st) {
  k_multiplier_full<<<1216, 256, 0, st>>>(dst, p->U0, p->g, p->n[0], p->n[1], p->n[2]);
  return cudaGetLastError();
}

template cudaError_t launch_atkm<double>(atkm_plan*, int, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_atkm<float>(atkm_plan*, int, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_H<double>(atkm_plan*, const Phys&, const double*, const double*, const double*, double*, int, cudaStream_t);
template cudaError_t launch_H<float>(atkm_plan*, const Phys&, const double*, const double*, const double*, double*, int, cudaStream_t);
template cudaError_t launch_precond<double>(atkm_plan*, const Phys&, const double*, const double*, const double*, const double*, double*, cudaStream_t);
template cudaError_t launch_precond<float>(atkm_plan*, const Phys&, const double*, const double*, const double*, const double*, double*, cudaStream_t);

}  // namespace atkm
