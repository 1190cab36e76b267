// Launchers of the three spectral operators for one arithmetic type R (the
// translation units passes_f64.cu and passes_f32.cu instantiate them).
#pragma once

#include <math.h>

#include "ops.cuh"

namespace atkm {

template <typename R> inline cx<R>* ws1(atkm_plan* p);
template <> inline double2* ws1<double>(atkm_plan* p) { return p->W1; }
template <> inline float2* ws1<float>(atkm_plan* p) { return p->W1f; }
// double-word passes reuse the FP64 workspaces (16-byte complex elements as well)
template <> inline cdf* ws1<df>(atkm_plan* p) { return reinterpret_cast<cdf*>(p->W1); }
template <typename R> inline cx<R>* ws2(atkm_plan* p);
template <> inline double2* ws2<double>(atkm_plan* p) { return p->W2; }
template <> inline float2* ws2<float>(atkm_plan* p) { return p->W2f; }
template <> inline cdf* ws2<df>(atkm_plan* p) { return reinterpret_cast<cdf*>(p->W2); }
template <typename R> inline cx<R>* ws3(atkm_plan* p);
template <> inline double2* ws3<double>(atkm_plan* p) { return p->T1; }
template <> inline float2* ws3<float>(atkm_plan* p) { return p->T1f; }
template <> inline cdf* ws3<df>(atkm_plan* p) { return reinterpret_cast<cdf*>(p->T1); }
// z-pass multiplier: the plan's table (FP64, double-word) or the U0 octant
// it is formed from in the pass (FP32); see OpAtkmZ.
template <typename R> inline const R* kztab(atkm_plan* p);
template <> inline const double* kztab<double>(atkm_plan* p) { return p->Kz; }
template <> inline const float* kztab<float>(atkm_plan* p) { return p->U0f; }
template <> inline const df* kztab<df>(atkm_plan* p) { return p->Kzd; }

template <typename R> inline const char* nm(const char* d, const char* f, const char* w) {
  return std::is_same<R, double>::value ? d : (std::is_same<R, float>::value ? f : w);
}
inline double fftflops(double n) { return 5.0 * n * log2(n); }

#define ATKM_RUN(NAME, BYTES, FLOPS, OP, FLEN, PG)              \
  do {                                                         \
    prof_begin(p, NAME, BYTES, FLOPS, st);                     \
    cudaError_t e_ = run_pass<R>(OP, FLEN, PG, st);            \
    prof_end(p, st);                                           \
    count_launches(1);                                         \
    if (e_ != cudaSuccess) return e_;                          \
  } while (0)

// The plan's tables of axis a (0, 1, 2 = x, y, z); see AxT.
inline AxT axt(const atkm_plan* p, int a) {
  const int Ns[3] = {p->g.Nx, p->g.Ny, p->g.Nz};
  size_t off = 0;
  for (int b = 0; b < a; ++b) off += 5 * (size_t)Ns[b];
  const double* t = p->axtab + off;
  const size_t n = (size_t)Ns[a];
  AxT r;
  r.nuN = t; r.kinN = t + n; r.hnu2 = t + 2 * n; r.xc = t + 3 * n; r.hxc2 = t + 4 * n;
  return r;
}

// What every ATKM pass needs of the plan: workspaces, constants, the byte and
// flop counts of the profiler.
template <typename R> struct AtkmCtx {
  const Geo* g;
  cx<R>* W1;
  cx<R>* W2;
  const R* K;
  Cst<R> c;
  const cx<R>* twM;
  double N, s, H1, fx, fy, fz, kb;
  long nl;
};
template <typename R> inline AtkmCtx<R> atkm_ctx(atkm_plan* p) {
  AtkmCtx<R> x;
  const Geo& g = p->g;
  x.g = &g;
  x.W1 = ws1<R>(p);
  x.W2 = ws2<R>(p);
  x.K = kztab<R>(p);
  x.c = make_cst<R>(g);
  x.twM = tw_table_host<R>(p->fM[0]);
  x.N = (double)g.Nx * g.Ny * g.Nz;
  x.s = (double)sizeof(cx<R>);
  x.H1 = (double)g.Nz * g.Ny * g.Xh;  // half-spectrum elements of W1
  x.fx = (double)g.Nz * g.Ny * fftflops(g.Nx);
  x.fy = (double)g.Nz * g.Xh * fftflops(g.My);
  x.fz = 2.0 * g.My * g.Xh * fftflops(g.Mz);
  // multiplier: the table read once, or the U0 octant
  x.kb = OpAtkmZ<R>::kTable ? (double)sizeof(R) * g.Mz * g.My * g.Xh
                            : (double)sizeof(R) * (g.Nx + 1) * (g.Ny + 1) * (g.Nz + 1);
  x.nl = (long)g.Nz * g.Ny;
  return x;
}

// The five passes of one ATKM evaluation, each a function of its own (same
// signature) so that heavy instantiations can compile in separate
// translation units.
// x forward (real data: complex FFT of length Nx + post-twist)
template <typename R>
cudaError_t atkm_pass_xf(atkm_plan* p, int mode, const double* a, const double* b, double*, cudaStream_t st) {
  const AtkmCtx<R> x = atkm_ctx<R>(p);
  const Geo& g = *x.g;
  if (!x.W1) return cudaErrorInvalidValue;
  const double inb = mode == SRC_RHO ? 8.0 : (mode == SRC_PSI ? 16.0 : 32.0);
  const PassGrid gx = pass_grid<R>(p, g.Nx, true, x.nl, 0, 0);
  const char* nx = nm<R>("atkm_x_fwd_f64", "atkm_x_fwd_f32", "atkm_x_fwd_df");
  if (mode == SRC_RHO) {
    OpAtkmXF<R, SRC_RHO> op; op.a = a; op.b = b; op.W1 = x.W1; op.twM = x.twM; op.c = x.c; op.XS = g.XS;
    ATKM_RUN(nx, inb * x.N + x.H1 * x.s, x.fx, op, p->fN[0], gx);
  } else if (mode == SRC_PSI) {
    OpAtkmXF<R, SRC_PSI> op; op.a = a; op.b = b; op.W1 = x.W1; op.twM = x.twM; op.c = x.c; op.XS = g.XS;
    ATKM_RUN(nx, inb * x.N + x.H1 * x.s, x.fx, op, p->fN[0], gx);
  } else {
    OpAtkmXF<R, SRC_PAIR> op; op.a = a; op.b = b; op.W1 = x.W1; op.twM = x.twM; op.c = x.c; op.XS = g.XS;
    ATKM_RUN(nx, inb * x.N + x.H1 * x.s, x.fx, op, p->fN[0], gx);
  }
  return cudaSuccess;
}

// y forward on the Nx + 1 half-spectrum columns
template <typename R>
cudaError_t atkm_pass_yf(atkm_plan* p, int, const double*, const double*, double*, cudaStream_t st) {
  const AtkmCtx<R> x = atkm_ctx<R>(p);
  const Geo& g = *x.g;
  if (!x.W1 || !x.W2) return cudaErrorInvalidValue;
  const PassGrid gy = pass_grid<R>(p, g.My, false, 0, g.Xh, g.Nz);
  OpAtkmYF<R> op; op.W1 = x.W1; op.W2 = x.W2; op.c = x.c; op.XS = g.XS;
  ATKM_RUN(nm<R>("atkm_y_fwd_f64", "atkm_y_fwd_f32", "atkm_y_fwd_df"), 3 * x.H1 * x.s, x.fy, op, p->fM[1], gy);
  return cudaSuccess;
}

// z forward * K_sym * inverse
template <typename R>
cudaError_t atkm_pass_z(atkm_plan* p, int, const double*, const double*, double*, cudaStream_t st) {
  const AtkmCtx<R> x = atkm_ctx<R>(p);
  const Geo& g = *x.g;
  if (!x.W2 || !x.K) return cudaErrorInvalidValue;
  OpAtkmZ<R> op; op.W2 = x.W2; op.K = x.K; op.U0 = x.K; op.c = x.c; op.XS = g.XS;
  op.n0 = (R)p->n[0]; op.n1 = (R)p->n[1]; op.n2 = (R)p->n[2];
  op.invM = (R)(0.5 / ((double)g.Mx * g.My * g.Mz));  // with the x forward pass's 1/2 (OpAtkmXF)
  const PassGrid pg = pass_grid<R>(p, g.Mz, false, 0, g.Xh, g.My);
  ATKM_RUN(nm<R>("atkm_z_f64", "atkm_z_f32", "atkm_z_df"), 4 * x.H1 * x.s + x.kb, x.fz, op, p->fM[2], pg);
  return cudaSuccess;
}

// y inverse
template <typename R>
cudaError_t atkm_pass_yi(atkm_plan* p, int, const double*, const double*, double*, cudaStream_t st) {
  const AtkmCtx<R> x = atkm_ctx<R>(p);
  const Geo& g = *x.g;
  if (!x.W1 || !x.W2) return cudaErrorInvalidValue;
  const PassGrid gy = pass_grid<R>(p, g.My, false, 0, g.Xh, g.Nz);
  OpAtkmYI<R> op; op.W2 = x.W2; op.W1 = x.W1; op.c = x.c; op.XS = g.XS;
  ATKM_RUN(nm<R>("atkm_y_inv_f64", "atkm_y_inv_f32", "atkm_y_inv_df"), 3 * x.H1 * x.s, x.fy, op, p->fM[1], gy);
  return cudaSuccess;
}

// x inverse (C2R) + crop
template <typename R>
cudaError_t atkm_pass_xi(atkm_plan* p, int, const double*, const double*, double* phi, cudaStream_t st) {
  const AtkmCtx<R> x = atkm_ctx<R>(p);
  const Geo& g = *x.g;
  if (!x.W1) return cudaErrorInvalidValue;
  const PassGrid gx = pass_grid<R>(p, g.Nx, true, x.nl, 0, 0);
  OpAtkmXI<R> op; op.W1 = x.W1; op.phi = phi; op.twM = x.twM; op.c = x.c; op.XS = g.XS;
  ATKM_RUN(nm<R>("atkm_x_inv_f64", "atkm_x_inv_f32", "atkm_x_inv_df"), x.H1 * x.s + 8 * x.N, x.fx, op, p->fN[0],
           gx);
  return cudaSuccess;
}

template <typename R>
cudaError_t launch_atkm(atkm_plan* p, int mode, const double* a, const double* b, double* phi, cudaStream_t st) {
  if (!ws1<R>(p) || !ws2<R>(p) || !kztab<R>(p)) return cudaErrorInvalidValue;
  cudaError_t e = atkm_pass_xf<R>(p, mode, a, b, phi, st);
  if (e == cudaSuccess) e = atkm_pass_yf<R>(p, mode, a, b, phi, st);
  if (e == cudaSuccess) e = atkm_pass_z<R>(p, mode, a, b, phi, st);
  if (e == cudaSuccess) e = atkm_pass_yi<R>(p, mode, a, b, phi, st);
  if (e == cudaSuccess) e = atkm_pass_xi<R>(p, mode, a, b, phi, st);
  return e;
}

// One axis pass of H_phi f (a function of its own so that heavy
// instantiations can be compiled in separate translation units).
template <typename R>
cudaError_t h_pass_x(atkm_plan* p, const Phys& ph, const double* f, const double* phi, const double* Phi, double* Hf,
                    int red_slot, cudaStream_t st) {
  const Geo& g = p->g;
  cx<R>* acc = ws3<R>(p);
  if (!acc) return cudaErrorInvalidValue;
  const bool red = red_slot >= 0;
  const Cst<R> c = make_cst<R>(g);
  const PhysR<R> pr = make_physr<R>(ph);
  const double2* fin = reinterpret_cast<const double2*>(f);
  const double2* pin = reinterpret_cast<const double2*>(phi);
  double2* out = reinterpret_cast<double2*>(Hf);
  const double N = (double)g.Nx * g.Ny * g.Nz, s = (double)sizeof(cx<R>);
  const long nl = (long)g.Nz * g.Ny;
  cudaError_t e;
  (void)pin; (void)out; (void)nl; (void)pr; (void)e;
  // x
  {
    const PassGrid pg = pass_grid<R>(p, g.Nx, true, nl, 0, 0);
    const double fl = 2.0 * nl * fftflops(g.Nx);
    const char* n = nm<R>("H_x_f64", "H_x_f32", "H_x_df");
    if (red) {
      OpHX<R, true> op; op.f = fin; op.acc = acc; op.c = c; op.Omega = pr.Omega; op.ax = axt(p, 0); op.ay = axt(p, 1);
      op.part = p->partials; op.pstride = pg.grid.x * pg.grid.y;
      ATKM_RUN(n, 16 * N + N * s, fl, op, p->fN[0], pg);
      if ((e = launch_finalize(p, 2, pg.grid.x * pg.grid.y, red_slot + 0, st)) != cudaSuccess) return e;
    } else {
      OpHX<R, false> op; op.f = fin; op.acc = acc; op.c = c; op.Omega = pr.Omega; op.ax = axt(p, 0); op.ay = axt(p, 1);
      ATKM_RUN(n, 16 * N + N * s, fl, op, p->fN[0], pg);
    }
  }
  return cudaSuccess;
}

template <typename R>
cudaError_t h_pass_y(atkm_plan* p, const Phys& ph, const double* f, const double* phi, const double* Phi, double* Hf,
                    int red_slot, cudaStream_t st) {
  const Geo& g = p->g;
  cx<R>* acc = ws3<R>(p);
  if (!acc) return cudaErrorInvalidValue;
  const bool red = red_slot >= 0;
  const Cst<R> c = make_cst<R>(g);
  const PhysR<R> pr = make_physr<R>(ph);
  const double2* fin = reinterpret_cast<const double2*>(f);
  const double2* pin = reinterpret_cast<const double2*>(phi);
  double2* out = reinterpret_cast<double2*>(Hf);
  const double N = (double)g.Nx * g.Ny * g.Nz, s = (double)sizeof(cx<R>);
  const long nl = (long)g.Nz * g.Ny;
  cudaError_t e;
  (void)pin; (void)out; (void)nl; (void)pr; (void)e;
  // y
  {
    const PassGrid pg = pass_grid<R>(p, g.Ny, false, 0, g.Nx, g.Nz);
    const double fl = 2.0 * g.Nz * g.Nx * fftflops(g.Ny);
    const char* n = nm<R>("H_y_f64", "H_y_f32", "H_y_df");
    if (red) {
      OpHY<R, true> op; op.f = fin; op.acc = acc; op.c = c; op.Omega = pr.Omega; op.ax = axt(p, 0); op.ay = axt(p, 1);
      op.part = p->partials; op.pstride = pg.grid.x * pg.grid.y;
      ATKM_RUN(n, 16 * N + 2 * N * s, fl, op, p->fN[1], pg);
      if ((e = launch_finalize(p, 2, pg.grid.x * pg.grid.y, red_slot + 2, st)) != cudaSuccess) return e;
    } else {
      OpHY<R, false> op; op.f = fin; op.acc = acc; op.c = c; op.Omega = pr.Omega; op.ax = axt(p, 0); op.ay = axt(p, 1);
      ATKM_RUN(n, 16 * N + 2 * N * s, fl, op, p->fN[1], pg);
    }
  }
  return cudaSuccess;
}

template <typename R>
cudaError_t h_pass_z(atkm_plan* p, const Phys& ph, const double* f, const double* phi, const double* Phi, double* Hf,
                    int red_slot, cudaStream_t st) {
  const Geo& g = p->g;
  cx<R>* acc = ws3<R>(p);
  if (!acc) return cudaErrorInvalidValue;
  const bool red = red_slot >= 0;
  const Cst<R> c = make_cst<R>(g);
  const PhysR<R> pr = make_physr<R>(ph);
  const double2* fin = reinterpret_cast<const double2*>(f);
  const double2* pin = reinterpret_cast<const double2*>(phi);
  double2* out = reinterpret_cast<double2*>(Hf);
  const double N = (double)g.Nx * g.Ny * g.Nz, s = (double)sizeof(cx<R>);
  const long nl = (long)g.Nz * g.Ny;
  cudaError_t e;
  (void)pin; (void)out; (void)nl; (void)pr; (void)e;
  // z + pointwise
  {
    const PassGrid pg = pass_grid<R>(p, g.Nz, false, 0, g.Nx, g.Ny);
    const double fl = 2.0 * g.Ny * g.Nx * fftflops(g.Nz);
    const char* n = nm<R>("H_z_f64", "H_z_f32", "H_z_df");
    if (red) {
      OpHZ<R, true> op; op.f = fin; op.phi = pin; op.Phi = Phi; op.acc = acc; op.Hf = out; op.c = c; op.ph = pr;
      op.ax = axt(p, 0); op.ay = axt(p, 1); op.az = axt(p, 2);
      op.same = fin == pin;
      op.part = p->partials; op.pstride = pg.grid.x * pg.grid.y;
      ATKM_RUN(n, (op.same ? 40 : 56) * N + N * s, fl, op, p->fN[2], pg);
      if ((e = launch_finalize(p, 6, pg.grid.x * pg.grid.y, red_slot + 4, st)) != cudaSuccess) return e;
    } else {
      OpHZ<R, false> op; op.f = fin; op.phi = pin; op.Phi = Phi; op.acc = acc; op.Hf = out; op.c = c; op.ph = pr;
      op.ax = axt(p, 0); op.ay = axt(p, 1); op.az = axt(p, 2);
      op.same = fin == pin;
      ATKM_RUN(n, (op.same ? 40 : 56) * N + N * s, fl, op, p->fN[2], pg);
    }
  }
  return cudaSuccess;
}

template <typename R>
cudaError_t launch_H(atkm_plan* p, const Phys& ph, const double* f, const double* phi, const double* Phi, double* Hf,
                     int red_slot, cudaStream_t st) {
  cudaError_t e = h_pass_x<R>(p, ph, f, phi, Phi, Hf, red_slot, st);
  if (e == cudaSuccess) e = h_pass_y<R>(p, ph, f, phi, Phi, Hf, red_slot, st);
  if (e == cudaSuccess) e = h_pass_z<R>(p, ph, f, phi, Phi, Hf, red_slot, st);
  return e;
}

template <typename R>
cudaError_t launch_precond(atkm_plan* p, const Phys& ph, const double* alpha_dev, const double* r, const double* phi,
                           const double* Phi, double* Pr, cudaStream_t st) {
  const Geo& g = p->g;
  cx<R>* Wk = ws3<R>(p);
  if (!Wk) return cudaErrorInvalidValue;
  const Cst<R> c = make_cst<R>(g);
  const PhysR<R> pr = make_physr<R>(ph);
  const double N = (double)g.Nx * g.Ny * g.Nz, s = (double)sizeof(cx<R>);
  const long nl = (long)g.Nz * g.Ny;
  const double fx = (double)nl * fftflops(g.Nx), fy = (double)g.Nz * g.Nx * fftflops(g.Ny);
  const PassGrid gx = pass_grid<R>(p, g.Nx, true, nl, 0, 0);
  const PassGrid gy = pass_grid<R>(p, g.Ny, false, 0, g.Nx, g.Nz);
  const PassGrid gz = pass_grid<R>(p, g.Nz, false, 0, g.Nx, g.Ny);
  {
    OpPXF<R> op; op.r = reinterpret_cast<const double2*>(r); op.phi = reinterpret_cast<const double2*>(phi);
    op.Phi = Phi; op.Wk = Wk; op.c = c; op.ph = pr; op.alpha = alpha_dev;
    op.ax = axt(p, 0); op.ay = axt(p, 1); op.az = axt(p, 2); op.Pw = p->Pw;
    // binary64 also writes the weights (8 B a point)
    const double by = (std::is_same<R, double>::value ? 48.0 : 40.0) * N + N * s;
    ATKM_RUN(nm<R>("P_x_fwd_f64", "P_x_fwd_f32", "P_x_fwd_df"), by, fx, op, p->fN[0], gx);
  }
  {
    OpPY<R, -1> op; op.Wk = Wk; op.c = c;
    ATKM_RUN(nm<R>("P_y_f64", "P_y_f32", "P_y_df"), 2 * N * s, fy, op, p->fN[1], gy);
  }
  {
    OpPZ<R> op; op.Wk = Wk; op.c = c; op.alpha = alpha_dev; op.ax = axt(p, 0); op.ay = axt(p, 1); op.az = axt(p, 2);
    ATKM_RUN(nm<R>("P_z_f64", "P_z_f32", "P_z_df"), 2 * N * s, 2.0 * g.Ny * g.Nx * fftflops(g.Nz), op, p->fN[2], gz);
  }
  {
    OpPY<R, 1> op; op.Wk = Wk; op.c = c;
    ATKM_RUN(nm<R>("P_y_f64", "P_y_f32", "P_y_df"), 2 * N * s, fy, op, p->fN[1], gy);
  }
  {
    OpPXI<R> op; op.Wk = Wk; op.phi = reinterpret_cast<const double2*>(phi); op.Phi = Phi;
    op.Pr = reinterpret_cast<double2*>(Pr); op.c = c; op.ph = pr; op.alpha = alpha_dev; op.Pw = p->Pw;
    // binary64 reads the stored weights (8 B) instead of phi and Phi (24 B)
    const double by = (std::is_same<R, double>::value ? 24.0 : 40.0) * N + N * s;
    ATKM_RUN(nm<R>("P_x_inv_f64", "P_x_inv_f32", "P_x_inv_df"), by, fx, op, p->fN[0], gx);
  }
  return cudaSuccess;
}

// In-place unnormalised 3D complex FFT (sign S) of buf on the plan's grid.
template <typename R>
cudaError_t launch_cfft3(atkm_plan* p, cx<R>* buf, int sign, cudaStream_t st) {
  const Geo& g = p->g;
  const Cst<R> c = make_cst<R>(g);
  const double N = (double)g.Nx * g.Ny * g.Nz, s = (double)sizeof(cx<R>);
  const long nl = (long)g.Nz * g.Ny;
  const PassGrid gx = pass_grid<R>(p, g.Nx, true, nl, 0, 0);
  const PassGrid gy = pass_grid<R>(p, g.Ny, false, 0, g.Nx, g.Nz);
  const PassGrid gz = pass_grid<R>(p, g.Nz, false, 0, g.Nx, g.Ny);
  const double fx = (double)nl * fftflops(g.Nx), fy = (double)g.Nz * g.Nx * fftflops(g.Ny),
               fz = (double)g.Ny * g.Nx * fftflops(g.Nz);
  if (sign < 0) {
    { OpCX<R, -1> op; op.buf = buf; op.c = c; ATKM_RUN("fft3_x", 2 * N * s, fx, op, p->fN[0], gx); }
    { OpPY<R, -1> op; op.Wk = buf; op.c = c; ATKM_RUN("fft3_y", 2 * N * s, fy, op, p->fN[1], gy); }
    { OpCZ<R, -1> op; op.buf = buf; op.c = c; ATKM_RUN("fft3_z", 2 * N * s, fz, op, p->fN[2], gz); }
  } else {
    { OpCX<R, 1> op; op.buf = buf; op.c = c; ATKM_RUN("fft3_x", 2 * N * s, fx, op, p->fN[0], gx); }
    { OpPY<R, 1> op; op.Wk = buf; op.c = c; ATKM_RUN("fft3_y", 2 * N * s, fy, op, p->fN[1], gy); }
    { OpCZ<R, 1> op; op.buf = buf; op.c = c; ATKM_RUN("fft3_z", 2 * N * s, fz, op, p->fN[2], gz); }
  }
  return cudaSuccess;
}

#undef ATKM_RUN

}  // namespace atkm
