// Fused tendency + RK3 substage update, and the eddy-diffusivity kernel.
//
// Physics (arXiv 2502.14148): flux-form advection (Eq. flux-form-advection,
// Eq. advection-flux-divergence) with WENO-Z reconstruction of the advected
// quantity (Eq. fifth-order-weno, order 2R-1) and, for momentum, a centered
// advecting velocity of order 2R-2 (Sec. B.2.1); closure fluxes (Sec. 3.1.1:
// ScalarDiffusivity in Laplacian form, Smagorinsky-Lilly / AMD in stress
// form); f-plane Coriolis; buoyancy b z_hat (Eq. buoyancy, linear EOS);
// prescribed top/bottom fluxes; finite-volume flux divergence
// (Eq. flux-divergence); RK3 substage (Eq. rk3).
//
// Kernel layout (GB300, one CTA per TX x TY column tile, marching up in z):
//  * The current level of every field, with an R-wide halo, is staged in
//    shared memory by cp.async (periodic wrap done by the gather), double or
//    triple buffered so that level k+1 streams in while level k is computed.
//  * Each thread also keeps its own column's 2R nearest levels of every field
//    in registers: the z-stencils come from there, with no shared traffic.
//  * Each thread computes the fluxes through the west, south and top faces of
//    its control volumes; the tile's east column and north row of faces are
//    computed by two "ghost" warps.  x/y fluxes meet through shared memory,
//    z fluxes are carried in registers from one level to the next, so every
//    face flux is reconstructed exactly once.
//  * The epilogue forms G, applies u~ = u + dt (gamma G - zeta G_prev) and
//    writes the new state and G (the G_prev of the next substage).
//  * FP32 Smagorinsky-Lilly and AMD kernels also compute the eddy
//    diffusivities, two levels ahead of the march, from planes staged four
//    levels ahead: each main thread its own cell (its column from its register
//    rings), the ghost warps the one-cell ring around the tile; no separate
//    closure kernel and no round trip through HBM (nu_e is still written out,
//    for readers outside the step).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "batch.cuh"
#include "ocn_internal.cuh"
#include "weno_coeffs.h"

namespace ocn {

// Each translation unit that includes this header owns its copy of the FP64 tables
// (no relocatable device code), uploaded by its own upload function; the FP32 kernels
// take their coefficients as compile-time constants (weno_coeffs.h).
static __constant__ WenoTables<double> cWd;

static cudaError_t upload_tables_here(const WenoTables<double>& t) {
  // Pack beta as upper triangle with doubled off-diagonal terms.
  WenoTables<double> d = t;
  for (int r = 1; r <= kMaxR; ++r)
    for (int s = 0; s < r; ++s) {
      for (int a = 0; a < r; ++a)
        for (int b = 0; b < r; ++b) d.beta[r][s][a][b] = (b > a) ? 2.0 * t.beta[r][s][a][b] : (b == a ? t.beta[r][s][a][b] : 0.0);
      for (int a = 0; a < r - 1; ++a)
        for (int b = 0; b < r - 1; ++b)
          d.dbeta[r][s][a][b] = (b > a) ? 2.0 * t.dbeta[r][s][a][b] : (b == a ? t.dbeta[r][s][a][b] : 0.0);
    }
  return cudaMemcpyToSymbol(cWd, &d, sizeof(d));
}

// f(std::integral_constant<int, i>) for i = 0 .. N-1: loops whose index must be a compile-time
// constant (the reconstruction coefficients below are selected by it).
template <class F, int... I>
__device__ __forceinline__ void sfor_seq(F&& f, std::integer_sequence<int, I...>) {
  (f(std::integral_constant<int, I>()), ...);
}
template <int N, class F>
__device__ __forceinline__ void sfor(F&& f) {
  sfor_seq(f, std::make_integer_sequence<int, N>());
}

// Reconstruction coefficients by compile-time index: FP32 as immediates (weno_coeffs.h), FP64
// from the long-double tables in constant memory.
template <typename T> struct Coef;
template <> struct Coef<float> {
  template <int r, int s, int a> static __device__ __forceinline__ float gqd() {
    constexpr float v = WenoGqD<float, r, s, a>::value;
    return v;
  }
  template <int r, int s, int a, int b> static __device__ __forceinline__ float db() {
    constexpr float v = WenoDb<float, r, s, a, b>::value;
    return v;
  }
  template <int r, int s> static __device__ __forceinline__ float d() {
    constexpr float v = WenoD<float, r, s>::value;
    return v;
  }
  template <int p, int n> static __device__ __forceinline__ float cen() {
    constexpr float v = WenoCen<float, p, n>::value;
    return v;
  }
};
template <> struct Coef<double> {
  template <int r, int s, int a> static __device__ __forceinline__ double gqd() { return cWd.gq[r][s][a] * cWd.d[r][s]; }
  template <int r, int s, int a, int b> static __device__ __forceinline__ double db() { return cWd.dbeta[r][s][a][b]; }
  template <int r, int s> static __device__ __forceinline__ double d() { return cWd.d[r][s]; }
  template <int p, int n> static __device__ __forceinline__ double cen() { return cWd.cen[p][n]; }
};

// The reciprocals of the WENO weights and of the AMD normalisations: the hardware approximation
// (at most 1 ulp off), issued as the bare instruction.  Every WENO argument is a positive
// indicator plus 1e-8 or a weight sum of at least 1; an AMD quotient is used only where its
// denominator (a sum of squared gradients) is positive.
__device__ __forceinline__ float rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

// WENO(2r-1) at the interface between s[r-1] and s[r] (s holds cells m-r .. m+r-1),
// upwinded by the sign of vel (the branch for vel >= 0 when vel == 0).
// Evaluated in difference form: with d_m = t_{m+1} - t_m in the upwind frame,
// each substencil value is t_{r-1} + (linear form in its r-1 differences) and
// each Jiang-Shu indicator a quadratic form in them (both exact rewritings of
// the cell-value forms, the tables derived on the host).  Mirroring the
// stencil for vel < 0 reverses and negates the differences; the indicators are
// even in d, so only the final correction carries the sign.  The substencil
// values are formed already multiplied by their linear weights d_k, so that the
// WENO-Z weight alpha_k = d_k (1 + (tau / (beta_k + eps))^2) enters the
// numerator as (1 + ratio^2) q_k d_k and the denominator as one FMA.
template <typename T, int r>
__device__ __forceinline__ T weno(const T* s, T vel) {
  const bool pos = vel >= T(0);
  if constexpr (r == 1) {
    return pos ? s[0] : s[1];
  } else {
    T ds[2 * r - 1];
#pragma unroll
    for (int n = 0; n < 2 * r - 1; ++n) ds[n] = s[n + 1] - s[n];
    T d[2 * r - 2];                       // |upwind-frame differences| up to a common sign
#pragma unroll
    for (int m = 0; m < 2 * r - 2; ++m) d[m] = pos ? ds[m] : ds[2 * r - 2 - m];
    const T ref = pos ? s[r - 1] : s[r];
    const T sgn = pos ? T(1) : T(-1);
    T q[r], b[r];
    sfor<r>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      T acc = Coef<T>::template gqd<r, k, 0>() * d[k];
      sfor<r - 2>([&](auto ac) {
        constexpr int a = decltype(ac)::value + 1;
        acc = fma(Coef<T>::template gqd<r, k, a>(), d[k + a], acc);
      });
      q[k] = acc;
      T bb = T(0);
      sfor<r - 1>([&](auto ac) {
        constexpr int a = decltype(ac)::value;
        T inner = Coef<T>::template db<r, k, a, a>() * d[k + a];
        sfor<r - 2 - a>([&](auto cc) {
          constexpr int c = decltype(cc)::value + a + 1;
          inner = fma(Coef<T>::template db<r, k, a, c>(), d[k + c], inner);
        });
        bb = fma(inner, d[k + a], bb);
      });
      b[k] = bb;
    });
    const T tau = fabs(b[0] - b[r - 1]);
    T num = T(0), den = T(0);
    sfor<r>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      const T ratio = tau * rcp(b[k] + T(1e-8));
      const T a1 = fma(ratio, ratio, T(1));         // alpha_k / d_k
      num = fma(a1, q[k], num);
      den = fma(Coef<T>::template d<r, k>(), a1, den);
    });
    return fma(sgn, num * rcp(den), ref);
  }
}

// Closure-flux arithmetic with every rounding spelled out (separate multiplies and adds, or
// explicit FMAs).  Plain multiplies and adds may be fused into FMAs by the code generator, and it
// makes that choice separately for every tile variant; spelling the rounding out keeps all
// variants bit-identical.
template <typename T> __device__ __forceinline__ T rmul(T a, T b);
template <> __device__ __forceinline__ float rmul<float>(float a, float b) { return __fmul_rn(a, b); }
template <> __device__ __forceinline__ double rmul<double>(double a, double b) { return __dmul_rn(a, b); }
template <typename T> __device__ __forceinline__ T radd(T a, T b);
template <> __device__ __forceinline__ float radd<float>(float a, float b) { return __fadd_rn(a, b); }
template <> __device__ __forceinline__ double radd<double>(double a, double b) { return __dadd_rn(a, b); }
template <typename T> __device__ __forceinline__ T rsub(T a, T b) { return radd<T>(a, -b); }
template <typename T> __device__ __forceinline__ T rfma(T a, T b, T c);
template <> __device__ __forceinline__ float rfma<float>(float a, float b, float c) { return __fmaf_rn(a, b, c); }
template <> __device__ __forceinline__ double rfma<double>(double a, double b, double c) { return __fma_rn(a, b, c); }
// F - c g, one rounding
template <typename T> __device__ __forceinline__ T rflux(T F, T c, T g) { return rfma<T>(-c, g, F); }
// F - 2 nu S with the strain S = ((x - y) r + g) / 2 (a difference quotient and a gradient):
// F - nu ((x - y) r + g)
template <typename T> __device__ __forceinline__ T rstress(T F, T nu, T x, T y, T r, T g) {
  return rfma<T>(-nu, rfma<T>(rsub<T>(x, y), r, g), F);
}
// (a + b + c + d) / 4 and (a + b) / 2
template <typename T> __device__ __forceinline__ T ravg4(T a, T b, T c, T d) {
  return rmul<T>(T(0.25), radd<T>(radd<T>(radd<T>(a, b), c), d));
}
template <typename T> __device__ __forceinline__ T ravg2(T a, T b) { return rmul<T>(T(0.5), radd<T>(a, b)); }

// Centered reconstruction of order 2p at the interface between s[p-1] and s[p].
template <typename T, int p>
__device__ __forceinline__ T centered(const T* s) {
  T acc = T(0);
  sfor<p>([&](auto nc) {
    constexpr int n = decltype(nc)::value;
    acc = fma(Coef<T>::template cen<p, n>(), s[n] + s[2 * p - 1 - n], acc);
  });
  return acc;
}

// Wall-reduced variants: a ring holding levels m-R .. m+R-1 around interface m.
template <typename T, int R>
__device__ __forceinline__ T weno_reduced(const T* ring, int r, T vel) {
  if (r >= R) return weno<T, R>(ring, vel);
  if constexpr (R > 4) { if (r == 4) return weno<T, 4>(ring + R - 4, vel); }
  if constexpr (R > 3) { if (r == 3) return weno<T, 3>(ring + R - 3, vel); }
  if constexpr (R > 2) { if (r == 2) return weno<T, 2>(ring + R - 2, vel); }
  if (r == 1) return weno<T, 1>(ring + R - 1, vel);
  return T(0);
}
// Centered interpolation at the interface between ring[R-1-SHIFT] and ring[R-SHIFT],
// of order 2p (p <= R-1), for a ring of 2R values.
template <typename T, int R, int SHIFT>
__device__ __forceinline__ T centered_reduced(const T* ring, int p) {
  constexpr int P = R - 1;
  if (p >= P) return centered<T, P>(ring + R - SHIFT - P);
  if constexpr (P > 3) { if (p == 3) return centered<T, 3>(ring + R - SHIFT - 3); }
  if constexpr (P > 2) { if (p == 2) return centered<T, 2>(ring + R - SHIFT - 2); }
  if constexpr (P > 1) { if (p == 1) return centered<T, 1>(ring + R - SHIFT - 1); }
  return T(0);
}

__device__ __forceinline__ void cp_async(void* smem, const void* gmem, int bytes) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (bytes == 4) asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
  else asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

template <typename T>
__device__ __forceinline__ T buoyancy(const TendencyArgs<T>& a, T c0, T c1) {
  return a.eos == OCN_EOS_LINEAR_TS ? a.g_alpha * (c0 - a.T0) - a.g_beta * (c1 - a.S0) : c0;
}

// Closure classes the FP32 kernels are compiled for: fluxes of a constant diffusivity (or none),
// Smagorinsky-Lilly, AMD; the FP64 kernels choose at run time (kClAny).  A fixed class lets the
// compiler drop the other closures' branches.
constexpr int kClAny = 0, kClScalar = 1, kClSmag = 2, kClAmd = 3;
inline int closure_class(int closure) {
  return closure == OCN_CLOSURE_SMAGORINSKY ? kClSmag : (closure == OCN_CLOSURE_AMD ? kClAmd : kClScalar);
}

template <int TX, int TY>
struct TileGeom {
  static constexpr int NMAIN = TX * TY;
  static constexpr int NTHREADS = ((TX * TY + TX + TY) + 31) / 32 * 32;
};

// Staging depth of the z march: levels (u, v, tracers) and w faces are prefetched LAL and LAW
// ahead of the level being computed, into LAL + 1 and LAW + 1 rotating plane slots.  The fused
// eddy diffusivities (FP32 Smagorinsky-Lilly and AMD) are computed two levels ahead and need the
// levels on either side of that, hence the deeper staging.
template <typename T, int CL>
struct MarchSlots {
  static constexpr bool FUSE = sizeof(T) == 4 && (CL == kClSmag || CL == kClAmd);
  static constexpr int LAL = FUSE ? 4 : 1, LAW = FUSE ? 4 : 2;
  static constexpr int NSL = LAL + 1, NSW = LAW + 1;
};

// PREG: keep this thread's gather offsets in registers for the whole march (FP32 launches whose
// register budget, 65536 / (threads x blocks per SM), is at least 128 a thread; below that, and in
// the FP64 kernels, the extra registers spill and the offsets are formed per level instead).
template <typename T, int TX, int TY, int MINB>
struct GatherInRegisters {
  static constexpr bool value = sizeof(T) == 4 && 65536 / (TileGeom<TX, TY>::NTHREADS * MINB) >= 128;
};

template <typename T, int R, int NTR, int TX, int TY, int CL, bool PREG>
__device__ __forceinline__ void tendency_body(const TendencyArgs<T>& a, const uint3 bid) {
  constexpr int P = R - 1;          // advecting-velocity half width
  constexpr int H = R;              // plane halo
  constexpr int PW = TX + 2 * H;
  constexpr int PH = TY + 2 * H;
  constexpr int PLANE = PW * PH;
  constexpr int NT_ = TileGeom<TX, TY>::NTHREADS;
  constexpr int FXS = TY * (TX + 1);
  constexpr int FYS = (TY + 1) * TX;
  typedef MarchSlots<T, CL> MS;
  constexpr bool FUSE = MS::FUSE;
  constexpr int LAL = MS::LAL, LAW = MS::LAW, NSL = MS::NSL, NSW = MS::NSW;

  const int Nx = a.Nx, Ny = a.Ny, Nz = a.Nz;
  constexpr int nt = NTR;
  constexpr int nf = 3 + nt;
  const size_t plane = (size_t)Nx * Ny;
  const bool stress = (CL == kClAny) ? (a.closure == OCN_CLOSURE_SMAGORINSKY || a.closure == OCN_CLOSURE_AMD)
                                      : (CL == kClSmag || CL == kClAmd);
  const bool amd = (CL == kClAny) ? (a.closure == OCN_CLOSURE_AMD) : (CL == kClAmd);
  const bool scalar = (CL == kClAny || CL == kClScalar) ? (a.closure == OCN_CLOSURE_SCALAR) : false;
  const T hPr = T(0.5) * a.inv_Pr;           // nu_e / (2 Pr) factor of a face-mean tracer diffusivity

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  T* sU = sm;                             // NSL slots (level k, prefetch; with FUSE levels k .. k+3, prefetch)
  T* sV = sU + NSL * PLANE;               // NSL slots
  T* sW = sV + NSL * PLANE;               // NSW slots (faces k, k+1, prefetch; with FUSE faces k .. k+3, prefetch)
  T* sC = sW + NSW * PLANE;               // nt x NSL slots
  T* sNu = sC + NSL * nt * PLANE;         // 4 slots (levels k-1, k, k+1, prefetch or, with FUSE, computed) if stress
  T* sK = sNu + (stress ? 4 : 0) * PLANE; // nt x 3 slots if amd
  T* FX = sK + (amd ? 3 * nt : 0) * PLANE;
  T* FY = FX + nf * FXS;
  T* PHs = FY + nf * FYS;                 // hydrostatic pressure anomaly, [TY+1][TX+1] (offset -1)
  int* gi_tab = reinterpret_cast<int*>(PHs + (TY + 1) * (TX + 1));
  int* gj_tab = gi_tab + PW;
  // with FUSE, per level l <= Nz: (C_s Delta_l)^2, 1/dz_c[l], 1/(4 dz_f[l]) (0 at the walls), dz_c[l]^2
  T* sLev = reinterpret_cast<T*>(gj_tab + PH);

  const int tid = threadIdx.x;
  const int i0 = bid.x * TX, j0 = bid.y * TY;
  const int Wt = min(TX, Nx - i0), Ht = min(TY, Ny - j0);

  // roles: main (TX*TY), north ghost row (TX), east ghost column (TY), idle
  int role, lx, ly;
  if (tid < TX * TY) { role = 0; lx = tid % TX; ly = tid / TX; }
  else if (tid < TX * TY + TX) { role = 1; lx = tid - TX * TY; ly = Ht; }
  else if (tid < TX * TY + TX + TY) { role = 2; lx = Wt; ly = tid - TX * TY - TX; }
  else { role = 3; lx = 0; ly = 0; }
  const bool active = (role == 0) ? (lx < Wt && ly < Ht) : (role == 1 ? lx < Wt : (role == 2 ? ly < Ht : false));
#if OCN_BOUNDS_CHECK
  if (role <= 2) {   // the stencil window of this thread's plane reads and its face-flux slots
    const int rc = (ly + H) * PW + (lx + H);
    (void)OCN_CHK(rc - R * PW - R, PLANE, a.oob, kOobPlane);
    (void)OCN_CHK(rc + (R - 1) * PW + R - 1, PLANE, a.oob, kOobPlane);
    if (active && role != 1) (void)OCN_CHK(ly * (TX + 1) + lx + (role == 0 ? 1 : 0), FXS, a.oob, kOobFlux);
    if (active && role != 2) (void)OCN_CHK(ly * TX + lx + (role == 0 ? TX : 0), FYS, a.oob, kOobFlux);
  }
#endif

  for (int e = tid; e < PW; e += NT_) { int g = (i0 + e - H) % Nx; gi_tab[e] = g < 0 ? g + Nx : g; }
  for (int e = tid; e < PH; e += NT_) { int g = (j0 + e - H) % Ny; gj_tab[e] = g < 0 ? g + Ny : g; }
  __syncthreads();

  // With PREG, this thread's gather offsets (plane elements tid + q NT_, periodic wrap through the
  // tables; the same for every field and level; 32-bit, as grids are created with Nx Ny < 2^31) are
  // formed once, so that a level's cp.async issue costs one add each; otherwise they are formed per
  // element and level.
  constexpr int NIT = (PLANE + NT_ - 1) / NT_;
  int goff[PREG ? NIT : 1];
#pragma unroll
  for (int q = 0; q < (PREG ? NIT : 1); ++q) {
    const int e = tid + q * NT_;
    goff[q] = 0;
    if (PREG && e < PLANE) {
      const int yy = e / PW, xx = e - yy * PW;
      goff[q] = gj_tab[yy] * Nx + gi_tab[xx];
    }
  }
  auto load_plane = [&](T* dst, const T* field, int level) {
    const T* base = field + (size_t)level * plane;
    if constexpr (PREG) {
#pragma unroll
      for (int q = 0; q < NIT; ++q) {
        const int e = tid + q * NT_;
        if (e < PLANE) cp_async(dst + e, base + OCN_CHK(goff[q], plane, a.oob, kOobGather), (int)sizeof(T));
      }
    } else {
      for (int e = tid; e < PLANE; e += NT_) {
        const int yy = e / PW, xx = e - yy * PW;
        cp_async(dst + e, base + OCN_CHK((size_t)gj_tab[yy] * Nx + gi_tab[xx], plane, a.oob, kOobGather), (int)sizeof(T));
      }
    }
  };
  auto load_level = [&](int k) {  // u, v, tracers at level k (slot k % NSL)
    if (k >= Nz) return;
    const int sl = k % NSL;
    load_plane(sU + sl * PLANE, a.cur.u, k);
    load_plane(sV + sl * PLANE, a.cur.v, k);
    for (int n = 0; n < nt; ++n) load_plane(sC + (n * NSL + sl) * PLANE, a.cur.c[n], k);
  };
  auto load_wface = [&](int f) { if (f <= Nz) load_plane(sW + (f % NSW) * PLANE, a.cur.w, f); };
  auto load_diff = [&](int l) {
    if (l < 0 || l >= Nz) return;
    if (FUSE) return;
    if (stress) load_plane(sNu + (l & 3) * PLANE, a.nu, l);
    if (amd) for (int n = 0; n < nt; ++n) load_plane(sK + (3 * n + l % 3) * PLANE, a.kap[n], l);
  };

  // own column (periodic)
  const int ci = (i0 + lx) % Nx, cj = (j0 + ly) % Ny;
  const size_t col = (size_t)cj * Nx + ci;
  auto ld_c = [&](const T* f, int level) -> T { return (level >= 0 && level < Nz) ? __ldg(f + (size_t)level * plane + col) : T(0); };
  // full tracer value: stored anomaly + the level's reference profile
  auto ld_tr = [&](int t, int level) -> T {
    if (level < 0 || level >= Nz) return T(0);
    const T ref = a.cref[t] ? __ldg(a.cref[t] + level) : T(0);
    return __ldg(a.cur.c[t] + (size_t)level * plane + col) + ref;
  };
  auto cref_at = [&](int t, int level) -> T { return a.cref[t] ? __ldg(a.cref[t] + level) : T(0); };
  auto ld_w = [&](int face) -> T { return (face >= 0 && face <= Nz) ? __ldg(a.cur.w + (size_t)face * plane + col) : T(0); };


  // register rings: level (or face) k+1-R+n at index n
  T ru[2 * R], rv[2 * R], rw[2 * R], rc[NTR][2 * R];
#pragma unroll
  for (int n = 0; n < 2 * R; ++n) {
    ru[n] = ld_c(a.cur.u, 1 - R + n);
    rv[n] = ld_c(a.cur.v, 1 - R + n);
    rw[n] = ld_w(1 - R + n);
  }
#pragma unroll
  for (int t = 0; t < NTR; ++t)
#pragma unroll
    for (int n = 0; n < 2 * R; ++n) rc[t][n] = ld_tr(t, 1 - R + n);

  // Eddy diffusivities of level L (Sec. 3.1.1 closure equation) from the staged planes of levels
  // L-1 .. L+1 and w faces L, L+1, with the velocity gradients at the centre as the closure kernel
  // forms them (each off-diagonal gradient the mean of its four edge differences, wall edges 0):
  //   Smagorinsky-Lilly  nu_e = (C_s Delta)^2 sqrt(max(|S|^2 - C_b N^2 / Pr, 0)), |S|^2 = 2 S_ij S_ij,
  //                      Delta = (dx dy dz_L)^(1/3), N^2 the mean of the two face gradients of b;
  //   AMD                nu_e = max(0, -C sum_m D_m^2 (d_m u_i)(d_m u_j) S_ij / |grad u|^2),
  //                      kappa_e = max(0, -C sum_m D_m^2 (d_m u_i)(d_m c)(d_i c) / |grad c|^2) per tracer,
  //                      tracer gradients centred (the mean of the two face differences).
  // The mean of four edge differences telescopes to half-sums of centred differences.  A main
  // thread computes its own cell, taking the point's own column (u, v, w, tracers at the levels
  // L-1 .. L+1) from its register rings; the ghost warps compute the ring of cells around the tile
  // from the planes, with the tracers' full values (stored anomaly + reference profile, the same
  // rounding as the rings).  Multiply-adds are explicit (never left to contraction), so that every
  // thread and every tile variant computes the same bits for the same point.
  struct NuCol { T u0, um, up, v0, vm, vp, w0, w1, c0, cm, cp, d0, dm, dp; };
  auto nu_point = [&](int L, int e, const NuCol& o, T* kap) -> T {
    T nu = T(0);
    if constexpr (FUSE) {
      const bool lo = L >= 1, hi = L + 1 < Nz;
      const int s0 = L % NSL;
      const T* U0 = sU + s0 * PLANE; const T* V0 = sV + s0 * PLANE;
      const T* W0 = sW + (L % NSW) * PLANE; const T* W1 = sW + ((L + 1) % NSW) * PLANE;
      const T* Um = sU + ((L + NSL - 1) % NSL) * PLANE; const T* Up = sU + ((L + 1) % NSL) * PLANE;
      const T* Vm = sV + ((L + NSL - 1) % NSL) * PLANE; const T* Vp = sV + ((L + 1) % NSL) * PLANE;
      // (C_s Delta)^2, 1/dz_c, 1/(4 dz_f) of faces L (and L+1 in the next entry), dz_c^2
      const T* lc = sLev + 4 * L;
      const T rdzc = lc[1], rzl4 = lo ? lc[2] : T(0), rzh4 = hi ? lc[4 + 2] : T(0);
      const T qx = T(0.25) * a.rdx, qy = T(0.25) * a.rdy;
      const T u1 = U0[e + 1], v1 = V0[e + PW];
      const T ux = (u1 - o.u0) * a.rdx, vy = (v1 - o.v0) * a.rdy, wz = (o.w1 - o.w0) * rdzc;
      const T uy = __fmul_rn(qy, (U0[e + PW] - U0[e - PW]) + (U0[e + 1 + PW] - U0[e + 1 - PW]));
      const T vx = __fmul_rn(qx, (V0[e + 1] - V0[e - 1]) + (V0[e + 1 + PW] - V0[e - 1 + PW]));
      const T wx = __fmul_rn(qx, (W0[e + 1] - W0[e - 1]) + (W1[e + 1] - W1[e - 1]));
      const T wy = __fmul_rn(qy, (W0[e + PW] - W0[e - PW]) + (W1[e + PW] - W1[e - PW]));
      const T su = o.u0 + u1, sv = o.v0 + v1;
      const T ul = lo ? su - (o.um + Um[e + 1]) : T(0), uh = hi ? (o.up + Up[e + 1]) - su : T(0);
      const T vl = lo ? sv - (o.vm + Vm[e + PW]) : T(0), vh = hi ? (o.vp + Vp[e + PW]) - sv : T(0);
      const T uz = __fmaf_rn(rzl4, ul, __fmul_rn(rzh4, uh));
      const T vz = __fmaf_rn(rzl4, vl, __fmul_rn(rzh4, vh));
      if constexpr (CL == kClSmag) {
        T bl = lo ? o.c0 - o.cm : T(0), bh = hi ? o.cp - o.c0 : T(0);
        if (a.eos == OCN_EOS_LINEAR_TS) {
          const T dl = lo ? o.d0 - o.dm : T(0), dh = hi ? o.dp - o.d0 : T(0);
          bl = __fmaf_rn(a.g_alpha, bl, -__fmul_rn(a.g_beta, dl));
          bh = __fmaf_rn(a.g_alpha, bh, -__fmul_rn(a.g_beta, dh));
        }
        // N^2 = (bl rdzf_L + bh rdzf_{L+1}) / 2, with the quarter-scaled reciprocals doubled
        const T N2 = __fmul_rn(T(2), __fmaf_rn(rzl4, bl, __fmul_rn(rzh4, bh)));
        const T a12 = uy + vx, a13 = uz + wx, a23 = vz + wy;       // 2 S_12, 2 S_13, 2 S_23
        const T dg = __fmaf_rn(wz, wz, __fmaf_rn(vy, vy, __fmul_rn(ux, ux)));
        const T od = __fmaf_rn(a23, a23, __fmaf_rn(a13, a13, __fmul_rn(a12, a12)));
        const T SS = __fmaf_rn(T(2), dg, od);                          // 2 S_ij S_ij
        const T ex = __fmaf_rn(-a.Cb * a.inv_Pr, N2, SS);
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(ex));
        nu = (SS > T(0) && ex > T(0)) ? lc[0] * r : T(0);
      } else {                                                           // AMD
        const T G[3][3] = {{ux, uy, uz}, {vx, vy, vz}, {wx, wy, wz}};
        const T D2[3] = {a.dx * a.dx, a.dy * a.dy, lc[3]};
        // (G G)[p][m], then num = sum_m D2_m sum_p G[p][m] (G G)[p][m] (g^T S g = g^T G g)
        T num = T(0), den = T(0);
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          T h = T(0);
#pragma unroll
          for (int p = 0; p < 3; ++p) {
            const T gg = __fmaf_rn(G[p][2], G[2][m], __fmaf_rn(G[p][1], G[1][m], __fmul_rn(G[p][0], G[0][m])));
            h = __fmaf_rn(G[p][m], gg, h);
          }
          num = __fmaf_rn(D2[m], h, num);
        }
#pragma unroll
        for (int p = 0; p < 3; ++p)
#pragma unroll
          for (int q = 0; q < 3; ++q) den = __fmaf_rn(G[p][q], G[p][q], den);
        const T nv = (-a.C_amd * num) * rcp(den);      // used only where den > 0
        nu = (den > T(0) && nv > T(0)) ? nv : T(0);
        const T rzl2 = T(2) * rzl4, rzh2 = T(2) * rzh4;                // 1/(2 dz_f) of the two faces
        const T hx = T(0.5) * a.rdx, hy = T(0.5) * a.rdy;
#pragma unroll
        for (int t = 0; t < NTR; ++t) {
          const T* C0 = sC + (t * NSL + s0) * PLANE;
          const T c0 = t == 0 ? o.c0 : o.d0, cm = t == 0 ? o.cm : o.dm, cp = t == 0 ? o.cp : o.dp;
          const T dc0 = __fmul_rn(hx, C0[e + 1] - C0[e - 1]);
          const T dc1 = __fmul_rn(hy, C0[e + PW] - C0[e - PW]);
          const T dc2 = __fmaf_rn(rzl2, lo ? c0 - cm : T(0), __fmul_rn(rzh2, hi ? cp - c0 : T(0)));
          const T dc[3] = {dc0, dc1, dc2};
          T cn = T(0);
#pragma unroll
          for (int m = 0; m < 3; ++m) {
            const T gd = __fmaf_rn(G[2][m], dc2, __fmaf_rn(G[1][m], dc1, __fmul_rn(G[0][m], dc0)));
            cn = __fmaf_rn(__fmul_rn(D2[m], dc[m]), gd, cn);
          }
          const T cd = __fmaf_rn(dc2, dc2, __fmaf_rn(dc1, dc1, __fmul_rn(dc0, dc0)));
          const T kv = (-a.C_amd * cn) * rcp(cd);      // used only where cd > 0
          kap[t] = (cd > T(0) && kv > T(0)) ? kv : T(0);
        }
      }
    }
    return nu;
  };
  // Eddy diffusivities of level L on the tile and the one-cell ring around it.  A main thread
  // computes its own cell, its column from the ring entries RI-1, RI, RI+1 (levels L-1, L, L+1; w
  // faces L, L+1 at RI, RI+1); the ghost threads compute the ring's 2 (TX + 2) + 2 TY points (from
  // index r0 in steps of nr).  With 4 i + 2 main warps (32 x 14), the SM's schedulers 0 and 1 hold
  // one main warp more than schedulers 2 and 3, which hold the two ghost warps (a third of the flux
  // work, no epilogue); the cells of the main warps 4 i and 4 i + 1 then go to the ghost threads
  // too (NDEL of them), which evens out the schedulers' work.  nu_e of cells inside the grid is
  // written to the arena as well.
  constexpr int MAINW = TX * TY / 32;
  constexpr bool DELEG = FUSE && (TX * TY) % 32 == 0 && MAINW % 4 == 2;
  constexpr int NDEL = DELEG ? 64 * ((MAINW + 2) / 4) : 0;
  const bool delegated = DELEG && role == 0 && ((tid >> 5) & 3) < 2;
  auto smag_nu = [&](int L, auto RIc, int r0, int nr) {
    if constexpr (FUSE) {
      constexpr int RI = decltype(RIc)::value;
      constexpr int t1 = NTR > 1 ? 1 : 0;
      T* nuS = sNu + (L & 3) * PLANE;
      if (role == 0 && !delegated) {
        const int e = (ly + H) * PW + (lx + H);
        NuCol o;
        o.u0 = ru[RI]; o.um = ru[RI - 1]; o.up = ru[RI + 1];
        o.v0 = rv[RI]; o.vm = rv[RI - 1]; o.vp = rv[RI + 1];
        o.w0 = rw[RI]; o.w1 = rw[RI + 1];
        o.c0 = rc[0][RI]; o.cm = rc[0][RI - 1]; o.cp = rc[0][RI + 1];
        o.d0 = rc[t1][RI]; o.dm = rc[t1][RI - 1]; o.dp = rc[t1][RI + 1];
        T kap[NTR];
        const T nu = nu_point(L, e, o, kap);
        nuS[e] = nu;
        if constexpr (CL == kClAmd) {
#pragma unroll
          for (int t = 0; t < NTR; ++t) sK[(3 * t + L % 3) * PLANE + e] = kap[t];
        }
        if (a.nu_out && active) a.nu_out[(size_t)L * plane + col] = nu;
      } else if (role != 0) {
        const int s0 = L % NSL, sm = (L + NSL - 1) % NSL, sp = (L + 1) % NSL;
        const T r00 = cref_at(0, L), r0m = L >= 1 ? cref_at(0, L - 1) : T(0), r0p = L + 1 < Nz ? cref_at(0, L + 1) : T(0);
        const T r10 = cref_at(t1, L), r1m = L >= 1 ? cref_at(t1, L - 1) : T(0), r1p = L + 1 < Nz ? cref_at(t1, L + 1) : T(0);
        const T* W0 = sW + (L % NSW) * PLANE; const T* W1 = sW + ((L + 1) % NSW) * PLANE;
        constexpr int NR = 2 * (TX + 2) + 2 * TY;
#pragma unroll 1
        for (int q = r0; q < NR + NDEL; q += nr) {
          int qx, qy;
          if (q < TX + 2) { qx = q - 1; qy = -1; }
          else if (q < 2 * (TX + 2)) { qx = q - (TX + 2) - 1; qy = TY; }
          else if (q < 2 * (TX + 2) + TY) { qx = -1; qy = q - 2 * (TX + 2); }
          else if (q < NR) { qx = TX; qy = q - 2 * (TX + 2) - TY; }
          else {                                   // a delegated cell of main warp 4 i or 4 i + 1
            const int d = q - NR, mt = 128 * (d >> 6) + (d & 63);
            qy = mt / TX; qx = mt - qy * TX;
          }
          const int e = (qy + H) * PW + (qx + H);
#if OCN_BOUNDS_CHECK
          (void)OCN_CHK(e - PW - 1, PLANE, a.oob, kOobPlane);
          (void)OCN_CHK(e + PW + 1, PLANE, a.oob, kOobPlane);
#endif
          NuCol o;
          o.u0 = sU[s0 * PLANE + e]; o.um = sU[sm * PLANE + e]; o.up = sU[sp * PLANE + e];
          o.v0 = sV[s0 * PLANE + e]; o.vm = sV[sm * PLANE + e]; o.vp = sV[sp * PLANE + e];
          o.w0 = W0[e]; o.w1 = W1[e];
          o.c0 = sC[s0 * PLANE + e] + r00; o.cm = sC[sm * PLANE + e] + r0m; o.cp = sC[sp * PLANE + e] + r0p;
          o.d0 = sC[(t1 * NSL + s0) * PLANE + e] + r10; o.dm = sC[(t1 * NSL + sm) * PLANE + e] + r1m;
          o.dp = sC[(t1 * NSL + sp) * PLANE + e] + r1p;
          T kap[NTR];
          const T nu = nu_point(L, e, o, kap);
          nuS[e] = nu;
          if constexpr (CL == kClAmd) {
#pragma unroll
            for (int t = 0; t < NTR; ++t) sK[(3 * t + L % 3) * PLANE + e] = kap[t];
          }
          if (q >= NR && a.nu_out && qx < Wt && qy < Ht)
            a.nu_out[(size_t)L * plane + (size_t)(j0 + qy) * Nx + (i0 + qx)] = nu;
        }
      }
    }
  };

  for (int l = 0; l < LAL; ++l) load_level(l);
  for (int f = 0; f < LAW; ++f) load_wface(f);
  load_diff(0);
  load_diff(1);
  cp_async_commit();
  if constexpr (FUSE) {
    for (int l = tid; l <= Nz; l += NT_) {
      T cd2 = T(0), rz = T(0), rf = T(0);
      if (l < Nz) {
        const T cd = a.Cs * cbrtf(a.dx * a.dy * __ldg(a.dzc + l));
        cd2 = cd * cd;
        rz = __ldg(a.rdzc + l);
      }
      if (l >= 1 && l < Nz) rf = T(0.25) * __ldg(a.rdzf + l);
      const T dz = (l < Nz) ? __ldg(a.dzc + l) : T(0);
      sLev[4 * l] = cd2; sLev[4 * l + 1] = rz; sLev[4 * l + 2] = rf; sLev[4 * l + 3] = dz * dz;
    }
  }
  cp_async_wait_all();
  __syncthreads();
  if constexpr (FUSE) {             // nu_e of the first two levels (rings hold levels 1-R .. R)
    smag_nu(0, std::integral_constant<int, R - 1>(), tid - TX * TY, NT_ - TX * TY);
    if (1 < Nz) smag_nu(1, std::integral_constant<int, R>(), tid - TX * TY, NT_ - TX * TY);
    __syncthreads();
  }

  // carried z fluxes through the bottom face of the current control volumes
  T fz_u = a.bot[0], fz_v = a.bot[1], fz_w = T(0);
  T fz_c[NTR];
#pragma unroll
  for (int t = 0; t < NTR; ++t) fz_c[t] = a.bot[2 + t];

  const int rowc = (ly + H) * PW + (lx + H);   // this thread's plane index

  // Hydrostatic split (Eq. pressure-decomposition), used when stepping: b leaves
  // the w equation and u, v feel -grad_h p_hy with d p_hy/dz = b.  p_hy is
  // integrated up each column along the z march from the buoyancy anomaly
  // relative to column (0,0), whose horizontally uniform part has no horizontal
  // gradient; the difference from the unsplit form is an exact discrete
  // gradient, removed by the projection.  Main threads integrate their own
  // column, the east ghosts the west halo column, the north ghosts the south
  // halo row.
  const bool split = (a.mode == 0);
  T phy = T(0), anom_prev = T(0);
  int hidx = -1, phw = -1;               // SMEM plane index of the integrated column, PH slot written
  if (role == 0) { hidx = rowc; phw = (active ? (ly + 1) * (TX + 1) + lx + 1 : -1); }
  else if (role == 2) { hidx = (ly + H) * PW + (H - 1); phw = (ly < Ht) ? (ly + 1) * (TX + 1) : -1; }
  else if (role == 1) { hidx = (H - 1) * PW + (lx + H); phw = (lx < Wt) ? lx + 1 : -1; }

  // Three segments of the z march: bottom levels, interior levels (every z
  // stencil at full order, no wall), top levels.  The segment loop is unrolled,
  // so the interior copy of the level body is compiled without wall branches.
  const int kb = min(R - 1, Nz);
  const int ke = max(kb, Nz - R);
#pragma unroll
  for (int seg = 0; seg < 3; ++seg) {
  const bool INT = (seg == 1);
  const int k0 = (seg == 0) ? 0 : (seg == 1 ? kb : ke);
  const int k1 = (seg == 0) ? kb : (seg == 1 ? ke : Nz);
  for (int k = k0; k < k1; ++k) {
    // ---- prefetch the planes LAL (levels) and LAW (faces) ahead
    load_level(k + LAL);
    load_wface(k + LAW);
    load_diff(k + 2);
    cp_async_commit();
    const int sk = k % NSL;                      // slot of level k
    // nu_e two levels ahead, for the fluxes of levels k+1 and k+2 (each main thread its own cell,
    // the ghost warps the ring around the tile); slot (k+2) & 3 held nu_e of level k-2, which no
    // thread reads at level k
    if constexpr (FUSE) {
      if (k + 2 < Nz) smag_nu(k + 2, std::integral_constant<int, R + 1>(), tid - TX * TY, NT_ - TX * TY);
    }
    // next ring entries (level k+1+R)
    T nu_ = ld_c(a.cur.u, k + 1 + R), nv_ = ld_c(a.cur.v, k + 1 + R), nw_ = ld_w(k + 1 + R);
    T nc_[NTR];
#pragma unroll
    for (int t = 0; t < NTR; ++t) nc_[t] = ld_tr(t, k + 1 + R);
    // G^{m-1} of this thread's points, loaded early (used by the update at the end of the level)
    T gp_u = T(0), gp_v = T(0), gp_w = T(0), gp_c[NTR];
#pragma unroll
    for (int t = 0; t < NTR; ++t) gp_c[t] = T(0);
    if (a.mode == 0 && a.dt_zeta != T(0) && role == 0 && active) {
      const size_t id = OCN_CHK((size_t)k * plane + col, (size_t)Nz * plane, a.oob, kOobGlobal);
      gp_u = a.G.u[id]; gp_v = a.G.v[id]; gp_w = a.G.w[id];
#pragma unroll
      for (int t = 0; t < NTR; ++t) gp_c[t] = a.G.c[t][id];
    }
    T crk[NTR];                                  // reference profile at this level
#pragma unroll
    for (int t = 0; t < NTR; ++t) crk[t] = cref_at(t, k);

    const T* pU = sU + sk * PLANE;
    const T* pV = sV + sk * PLANE;
    const T* pW0 = sW + (k % NSW) * PLANE;        // face k
    const T* pW1 = sW + ((k + 1) % NSW) * PLANE;  // face k+1
    const T* pNm = sNu + ((k + 3) & 3) * PLANE; // level k-1
    const T* pN0 = sNu + (k & 3) * PLANE;       // level k
    const T* pN1 = sNu + ((k + 1) & 3) * PLANE; // level k+1
    const T rdzc_k = __ldg(a.rdzc + k);
    const T rdzf_k = (INT || k >= 1) ? __ldg(a.rdzf + k) : T(0);
    const T rdzf_k1 = (k + 1 < Nz) ? __ldg(a.rdzf + k + 1) : T(0);
    const T rdx = a.rdx, rdy = a.rdy;

    // ================= x fluxes (main threads and the east ghost column)
    if (role == 0 || role == 2) {
      T s[2 * R];
      // u: advecting U = centered_x(u), advected WENO_x(u), interface lx (centre lx-1)
#pragma unroll
      for (int n = 0; n < 2 * R; ++n) s[n] = pU[rowc - R + n];
      {
        const T U = centered<T, P>(s + R - P);
        T F = U * weno<T, R>(s, U);
        const T du = (s[R] - s[R - 1]) * rdx;
        if (scalar) F = rflux<T>(F, a.nu0, du);
        else if (stress) F = rflux<T>(F, rmul<T>(T(2), pN0[rowc - 1]), du);
        if (active) FX[0 * FXS + ly * (TX + 1) + lx] = F;
      }
      // v at (face i, face j): advecting centered_y(u), advected WENO_x(v)
      {
        T cu[2 * P];
#pragma unroll
        for (int n = 0; n < 2 * P; ++n) cu[n] = pU[rowc + (n - P) * PW];
        const T U = centered<T, P>(cu);
        T sv[2 * R];
#pragma unroll
        for (int n = 0; n < 2 * R; ++n) sv[n] = pV[rowc - R + n];
        T F = U * weno<T, R>(sv, U);
        const T dvdx = (sv[R] - sv[R - 1]) * rdx;
        if (scalar) F = rflux<T>(F, a.nu0, dvdx);
        else if (stress) {
          const T nuf = ravg4<T>(pN0[rowc - 1 - PW], pN0[rowc - PW], pN0[rowc - 1], pN0[rowc]);
          F = rstress<T>(F, nuf, pU[rowc], pU[rowc - PW], rdy, dvdx);
        }
        if (active) FX[1 * FXS + ly * (TX + 1) + lx] = F;
      }
      // w at (face i, face k): advecting centered_z(u) (own column), advected WENO_x(w)
      {
        T F = T(0);
        if (INT || k >= 1) {
          const int p = INT ? P : min(P, min(k, Nz - k));
          const T U = centered_reduced<T, R, 1>(ru, p);   // ru-1: levels k-R .. k+R-1 around face k
          T sw[2 * R];
#pragma unroll
          for (int n = 0; n < 2 * R; ++n) sw[n] = pW0[rowc - R + n];
          F = U * weno<T, R>(sw, U);
          const T dwdx = (sw[R] - sw[R - 1]) * rdx;
          if (scalar) F = rflux<T>(F, a.nu0, dwdx);
          else if (stress) {
            const T nuf = ravg4<T>(pNm[rowc - 1], pNm[rowc], pN0[rowc - 1], pN0[rowc]);
            F = rstress<T>(F, nuf, ru[R - 1], ru[R - 2], rdzf_k, dwdx);
          }
        }
        if (active) FX[2 * FXS + ly * (TX + 1) + lx] = F;
      }
      // tracers at face i: U = u, advected WENO_x(c)
#pragma unroll
      for (int t = 0; t < NTR; ++t) {
        const T* pC = sC + (t * NSL + sk) * PLANE;
        T sc[2 * R];
#pragma unroll
        for (int n = 0; n < 2 * R; ++n) sc[n] = pC[rowc - R + n];
        const T U = pU[rowc];
        T F = U * (weno<T, R>(sc, U) + crk[t]);    // reconstruction commutes with the level's constant shift
        const T dc = (sc[R] - sc[R - 1]) * rdx;
        if (scalar) F = rflux<T>(F, a.kappa0, dc);
        else if (amd) { const T* pK = sK + (3 * t + k % 3) * PLANE; F = rflux<T>(F, ravg2<T>(pK[rowc - 1], pK[rowc]), dc); }
        else if (stress) F = rflux<T>(F, rmul<T>(hPr, radd<T>(pN0[rowc - 1], pN0[rowc])), dc);
        if (active) FX[(3 + t) * FXS + ly * (TX + 1) + lx] = F;
      }
    }

    // ================= y fluxes (main threads and the north ghost row)
    if (role == 0 || role == 1) {
      // u at (face i, face j): advecting centered_x(v), advected WENO_y(u)
      {
        T cv[2 * P];
#pragma unroll
        for (int n = 0; n < 2 * P; ++n) cv[n] = pV[rowc - P + n];
        const T V = centered<T, P>(cv);
        T su[2 * R];
#pragma unroll
        for (int n = 0; n < 2 * R; ++n) su[n] = pU[rowc + (n - R) * PW];
        T F = V * weno<T, R>(su, V);
        const T dudy = (su[R] - su[R - 1]) * rdy;
        if (scalar) F = rflux<T>(F, a.nu0, dudy);
        else if (stress) {
          const T nuf = ravg4<T>(pN0[rowc - 1 - PW], pN0[rowc - PW], pN0[rowc - 1], pN0[rowc]);
          F = rstress<T>(F, nuf, pV[rowc], pV[rowc - 1], rdx, dudy);
        }
        if (active) FY[0 * FYS + ly * TX + lx] = F;
      }
      // v: advecting centered_y(v), advected WENO_y(v), interface ly (centre ly-1)
      {
        T sv[2 * R];
#pragma unroll
        for (int n = 0; n < 2 * R; ++n) sv[n] = pV[rowc + (n - R) * PW];
        const T V = centered<T, P>(sv + R - P);
        T F = V * weno<T, R>(sv, V);
        const T dv = (sv[R] - sv[R - 1]) * rdy;
        if (scalar) F = rflux<T>(F, a.nu0, dv);
        else if (stress) F = rflux<T>(F, rmul<T>(T(2), pN0[rowc - PW]), dv);
        if (active) FY[1 * FYS + ly * TX + lx] = F;
      }
      // w at (face j, face k): advecting centered_z(v) (own column), advected WENO_y(w)
      {
        T F = T(0);
        if (INT || k >= 1) {
          const int p = INT ? P : min(P, min(k, Nz - k));
          const T V = centered_reduced<T, R, 1>(rv, p);
          T sw[2 * R];
#pragma unroll
          for (int n = 0; n < 2 * R; ++n) sw[n] = pW0[rowc + (n - R) * PW];
          F = V * weno<T, R>(sw, V);
          const T dwdy = (sw[R] - sw[R - 1]) * rdy;
          if (scalar) F = rflux<T>(F, a.nu0, dwdy);
          else if (stress) {
            const T nuf = ravg4<T>(pNm[rowc - PW], pNm[rowc], pN0[rowc - PW], pN0[rowc]);
            F = rstress<T>(F, nuf, rv[R - 1], rv[R - 2], rdzf_k, dwdy);
          }
        }
        if (active) FY[2 * FYS + ly * TX + lx] = F;
      }
#pragma unroll
      for (int t = 0; t < NTR; ++t) {
        const T* pC = sC + (t * NSL + sk) * PLANE;
        T sc[2 * R];
#pragma unroll
        for (int n = 0; n < 2 * R; ++n) sc[n] = pC[rowc + (n - R) * PW];
        const T V = pV[rowc];
        T F = V * (weno<T, R>(sc, V) + crk[t]);
        const T dc = (sc[R] - sc[R - 1]) * rdy;
        if (scalar) F = rflux<T>(F, a.kappa0, dc);
        else if (amd) { const T* pK = sK + (3 * t + k % 3) * PLANE; F = rflux<T>(F, ravg2<T>(pK[rowc - PW], pK[rowc]), dc); }
        else if (stress) F = rflux<T>(F, rmul<T>(hPr, radd<T>(pN0[rowc - PW], pN0[rowc])), dc);
        if (active) FY[(3 + t) * FYS + ly * TX + lx] = F;
      }
    }

    // ================= z fluxes through the top faces (main threads), registers only
    T nz_u = T(0), nz_v = T(0), nz_w = T(0);
    T nz_c[NTR];
#pragma unroll
    for (int t = 0; t < NTR; ++t) nz_c[t] = T(0);
    if (role == 0) {
      const bool top = !INT && (k + 1 == Nz);
      const int r = INT ? R : min(R, min(k + 1, Nz - k - 1));        // centre fields at face k+1
      // u at (face i, face k+1): advecting centered_x(w at face k+1)
      if (top) nz_u = a.top[0];
      else {
        T cw[2 * P];
#pragma unroll
        for (int n = 0; n < 2 * P; ++n) cw[n] = pW1[rowc - P + n];
        const T Wv = centered<T, P>(cw);
        T F = Wv * weno_reduced<T, R>(ru, r, Wv);
        const T dudz = (ru[R] - ru[R - 1]) * rdzf_k1;
        if (scalar) F = rflux<T>(F, a.nu0, dudz);
        else if (stress) {
          const T nuf = ravg4<T>(pN0[rowc - 1], pN0[rowc], pN1[rowc - 1], pN1[rowc]);
          F = rstress<T>(F, nuf, pW1[rowc], pW1[rowc - 1], rdx, dudz);
        }
        nz_u = F;
      }
      if (top) nz_v = a.top[1];
      else {
        T cw[2 * P];
#pragma unroll
        for (int n = 0; n < 2 * P; ++n) cw[n] = pW1[rowc + (n - P) * PW];
        const T Wv = centered<T, P>(cw);
        T F = Wv * weno_reduced<T, R>(rv, r, Wv);
        const T dvdz = (rv[R] - rv[R - 1]) * rdzf_k1;
        if (scalar) F = rflux<T>(F, a.nu0, dvdz);
        else if (stress) {
          const T nuf = ravg4<T>(pN0[rowc - PW], pN0[rowc], pN1[rowc - PW], pN1[rowc]);
          F = rstress<T>(F, nuf, pW1[rowc], pW1[rowc - PW], rdy, dvdz);
        }
        nz_v = F;
      }
#pragma unroll
      for (int t = 0; t < NTR; ++t) {
        if (top) { nz_c[t] = a.top[2 + t]; continue; }
        const T Wv = rw[R];
        T F = Wv * weno_reduced<T, R>(rc[t], r, Wv);
        const T dc = (rc[t][R] - rc[t][R - 1]) * rdzf_k1;
        if (scalar) F = rflux<T>(F, a.kappa0, dc);
        else if (amd) {
          const T* pK0 = sK + (3 * t + k % 3) * PLANE;
          const T* pK1 = sK + (3 * t + (k + 1) % 3) * PLANE;
          F = rflux<T>(F, ravg2<T>(pK0[rowc], pK1[rowc]), dc);
        } else if (stress) F = rflux<T>(F, rmul<T>(hPr, radd<T>(pN0[rowc], pN1[rowc])), dc);
        nz_c[t] = F;
      }
      // w through centre k (w interface k+1; valid faces 0..Nz)
      {
        const int rw_ = INT ? R : min(R, min(k + 1, Nz - k));
        const int pw_ = INT ? P : min(P, min(k + 1, Nz - k));
        const T Wv = centered_reduced<T, R, 0>(rw, pw_);
        T F = Wv * weno_reduced<T, R>(rw, rw_, Wv);
        const T dw = (rw[R] - rw[R - 1]) * rdzc_k;
        if (scalar) F = rflux<T>(F, a.nu0, dw);
        else if (stress) F = rflux<T>(F, rmul<T>(T(2), pN0[rowc]), dw);
        nz_w = F;
      }
    }

    if (split && hidx >= 0) {
      const T* pC0 = sC + sk * PLANE;
      const T* pC1 = sC + ((NTR > 1 ? 1 : 0) * NSL + sk) * PLANE;
      constexpr int t1 = NTR > 1 ? 1 : 0;
      const T bref = buoyancy(a, __ldg(a.cur.c[0] + (size_t)k * plane) + crk[0], __ldg(a.cur.c[t1] + (size_t)k * plane) + crk[t1]);
      const T bhere = (role == 0) ? buoyancy(a, rc[0][R - 1], rc[t1][R - 1])
                                  : buoyancy(a, pC0[hidx] + crk[0], pC1[hidx] + crk[t1]);
      const T anom = bhere - bref;
      if (INT || k >= 1) phy = fma(__ldg(a.dzf + k) * T(0.5), anom_prev + anom, phy);
      anom_prev = anom;
      if (phw >= 0) PHs[phw] = phy;
    }

    __syncthreads();

    // ================= tendencies and RK update
    if (role == 0 && active) {
      const size_t id = OCN_CHK((size_t)k * plane + col, (size_t)Nz * plane, a.oob, kOobGlobal);
      const T* FXu = FX + ly * (TX + 1) + lx;
      const T* FYu = FY + ly * TX + lx;
      // u
      {
        const T vbar = T(0.25) * (pV[rowc - 1] + pV[rowc] + pV[rowc - 1 + PW] + pV[rowc + PW]);
        T G = -(FXu[1] - FXu[0]) * rdx - (FYu[TX] - FYu[0]) * rdy - (nz_u - fz_u) * rdzc_k + a.f * vbar;
        if (split) G -= (PHs[(ly + 1) * (TX + 1) + lx + 1] - PHs[(ly + 1) * (TX + 1) + lx]) * rdx;
        if (a.mode == 0) {
          T upd = fma(a.dt_gamma, G, ru[R - 1]);
          if (a.dt_zeta != T(0)) upd = fma(-a.dt_zeta, gp_u, upd);
          a.nxt.u[id] = upd;
        }
        a.G.u[id] = G;
      }
      // v
      {
        const T ubar = T(0.25) * (pU[rowc - PW] + pU[rowc + 1 - PW] + pU[rowc] + pU[rowc + 1]);
        T G = -(FXu[FXS + 1] - FXu[FXS]) * rdx - (FYu[FYS + TX] - FYu[FYS]) * rdy - (nz_v - fz_v) * rdzc_k - a.f * ubar;
        if (split) G -= (PHs[(ly + 1) * (TX + 1) + lx + 1] - PHs[ly * (TX + 1) + lx + 1]) * rdy;
        if (a.mode == 0) {
          T upd = fma(a.dt_gamma, G, rv[R - 1]);
          if (a.dt_zeta != T(0)) upd = fma(-a.dt_zeta, gp_v, upd);
          a.nxt.v[id] = upd;
        }
        a.G.v[id] = G;
      }
      // w at face k
      {
        T G = T(0);
        if (INT || k >= 1) {
          G = -(FXu[2 * FXS + 1] - FXu[2 * FXS]) * rdx - (FYu[2 * FYS + TX] - FYu[2 * FYS]) * rdy
              - (nz_w - fz_w) * rdzf_k;
          if (!split) {   // unsplit form (tendency output): + b interpolated to the w face
            const T bk = buoyancy(a, rc[0][R - 1], rc[NTR > 1 ? 1 : 0][R - 1]);
            const T bkm = buoyancy(a, rc[0][R - 2], rc[NTR > 1 ? 1 : 0][R - 2]);
            G += T(0.5) * (bkm + bk);
          }
        }
        if (a.mode == 0) {
          T upd = T(0);
          if (INT || k >= 1) {
            upd = fma(a.dt_gamma, G, rw[R - 1]);
            if (a.dt_zeta != T(0)) upd = fma(-a.dt_zeta, gp_w, upd);
          }
          a.nxt.w[id] = upd;
          if (!INT && k == Nz - 1) a.nxt.w[id + plane] = T(0);
        }
        a.G.w[id] = G;
        if (!INT && k == Nz - 1) a.G.w[id + plane] = T(0);
      }
#pragma unroll
      for (int t = 0; t < NTR; ++t) {
        T G = -(FXu[(3 + t) * FXS + 1] - FXu[(3 + t) * FXS]) * rdx - (FYu[(3 + t) * FYS + TX] - FYu[(3 + t) * FYS]) * rdy
              - (nz_c[t] - fz_c[t]) * rdzc_k;
        if (a.mode == 0) {
          T upd = fma(a.dt_gamma, G, sC[(t * NSL + sk) * PLANE + rowc]);   // the stored anomaly
          if (a.dt_zeta != T(0)) upd = fma(-a.dt_zeta, gp_c[t], upd);
          a.nxt.c[t][id] = upd;
        }
        a.G.c[t][id] = G;
      }
    }

    // ---- advance: carry z fluxes, shift rings
    fz_u = nz_u; fz_v = nz_v; fz_w = nz_w;
#pragma unroll
    for (int t = 0; t < NTR; ++t) fz_c[t] = nz_c[t];
#pragma unroll
    for (int n = 0; n < 2 * R - 1; ++n) { ru[n] = ru[n + 1]; rv[n] = rv[n + 1]; rw[n] = rw[n + 1]; }
    ru[2 * R - 1] = nu_; rv[2 * R - 1] = nv_; rw[2 * R - 1] = nw_;
#pragma unroll
    for (int t = 0; t < NTR; ++t) {
#pragma unroll
      for (int n = 0; n < 2 * R - 1; ++n) rc[t][n] = rc[t][n + 1];
      rc[t][2 * R - 1] = nc_[t];
    }
    cp_async_wait_all();
    __syncthreads();
  }
  }
}

template <typename T, int R, int NTR, int TX, int TY, int MINB, int CL>
struct TendencyK {
  typedef TendencyArgs<T> Payload;
  static constexpr int kThreads = TileGeom<TX, TY>::NTHREADS, kMinBlocks = MINB;
  static __device__ __forceinline__ void run(const Payload& a, uint3 bid, uint3) {
    tendency_body<T, R, NTR, TX, TY, CL, GatherInRegisters<T, TX, TY, MINB>::value>(a, bid);
  }
};

template <typename T, int R, int NTR, int TX, int TY, int MINB, int CL>
__global__ void __launch_bounds__(TileGeom<TX, TY>::NTHREADS, MINB) k_tendency(const TendencyArgs<T> a) {
  tendency_body<T, R, NTR, TX, TY, CL, GatherInRegisters<T, TX, TY, MINB>::value>(a, blockIdx);
}

// The batched twin of k_tendency<T, R, NTR, TX, TY, MINB, CL> (k_batched over TendencyK),
// instantiated in the *_batch translation units so that the plain and batched kernels compile in
// parallel.
template <typename T, int R, int NTR, int TX, int TY, int MINB, int CL>
const void* tendency_batched_kernel();

// The FP32 tile variants (TX, TY, CTAs per SM), in the order of the variant index.
#define OCN_F32_TILE_VARIANTS(X, R, NTR, CL) \
  X(R, NTR, 32, 8, 1, CL) X(R, NTR, 32, 8, 2, CL) X(R, NTR, 32, 16, 1, CL) X(R, NTR, 32, 4, 3, CL) \
  X(R, NTR, 32, 14, 1, CL) X(R, NTR, 32, 12, 1, CL) X(R, NTR, 16, 16, 2, CL)

template <typename T, int R, int TX, int TY, int CL>
static size_t tendency_smem(const TendencyArgs<T>& a) {
  constexpr int H = R;
  constexpr int PLANE = (TX + 2 * H) * (TY + 2 * H);
  typedef MarchSlots<T, CL> MS;
  const bool stress = (a.closure == OCN_CLOSURE_SMAGORINSKY || a.closure == OCN_CLOSURE_AMD);
  const bool amd = (a.closure == OCN_CLOSURE_AMD);
  const int nf = 3 + a.nt;
  size_t planes = MS::NSL * (2 + a.nt) + MS::NSW + (stress ? 4 : 0) + (amd ? 3 * a.nt : 0);
  size_t bytes = sizeof(T) * (planes * PLANE + (size_t)nf * (TY * (TX + 1) + (TY + 1) * TX));
  bytes += sizeof(T) * (TY + 1) * (TX + 1);
  bytes += sizeof(int) * ((TX + 2 * H) + (TY + 2 * H));
  if (MS::FUSE) bytes += sizeof(T) * 4 * ((size_t)a.Nz + 1);
  return bytes;
}

// Launch one tile variant (TX x TY columns per CTA, at least MINB CTAs per SM) of closure class
// CL.  Instantiated explicitly, one closure class per translation unit.
template <typename T, int R, int NTR, int TX, int TY, int MINB, int CL>
cudaError_t launch_tendency_variant(const TendencyArgs<T>& a, cudaStream_t s) {
  auto kern = k_tendency<T, R, NTR, TX, TY, MINB, CL>;
  size_t smem = tendency_smem<T, R, TX, TY, CL>(a);
  cudaError_t e = raise_smem_limit(kern, smem);
  if (e != cudaSuccess) return e;
  if (MINB > 1) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((a.Nx + TX - 1) / TX, (a.Ny + TY - 1) / TY);
  if (LaunchRecorder* r = active_recorder()) {
    LaunchRecord rec;
    rec.fn = tendency_batched_kernel<T, R, NTR, TX, TY, MINB, CL>();
    rec.grid = grid;
    rec.block = dim3(TileGeom<TX, TY>::NTHREADS);
    rec.smem = smem;
    rec.kclass = OCN_K_TENDENCY;
    rec.carveout = MINB > 1 ? 100 : -1;
    rec.payload.assign(batch_stride(sizeof(a)), 0);
    memcpy(rec.payload.data(), &a, sizeof(a));
    r->list.push_back(std::move(rec));
    return cudaSuccess;
  }
  kern<<<grid, TileGeom<TX, TY>::NTHREADS, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace ocn
