// Pressure projection (Appendix A.2): rhs = div(u~)/dt, lap p = rhs solved by
// the eigenfunction expansion of the discrete Laplacian -- FFT in the periodic,
// equispaced x and y directions and a tridiagonal (Thomas) solve down each
// vertical column of the possibly stretched z grid -- then u = u~ - dt grad p
// (Eqs. pressure-poisson, pressure-correction).
//
// Kernels:
//   k_div_fftx : divergence of each x-row fused with its real-to-complex FFT
//                (half-length complex FFT + split), written to the half
//                spectrum [Nz][Ny][Sp] (kx = 0 .. Nx/2 of rows of stride Sp);
//   k_fft_y    : complex FFT along y for tiles of kx columns (forward/inverse);
//   k_tridiag  : one thread per (kx, ky) column; coalesced across kx;
//                Neumann walls; the (0,0) mode is pinned by p_0 = 0;
//   k_gauge    : one warp removes the volume mean of the (0,0) column;
//   k_ifftx    : complex-to-real inverse FFT along x -> p;
//   k_correct  : u -= dt grad p on every non-wall face.
// FFTs are shared-memory Stockham passes of radix 8/4/2/3 with host-built
// twiddle tables, so every size 2^a 3^b is handled.
#include <cuda_runtime.h>

#include <type_traits>

#include "batch.cuh"
#include "ocn_internal.cuh"

namespace ocn {

template <typename T> struct CT;
template <> struct CT<float> { typedef float2 type; };
template <> struct CT<double> { typedef double2 type; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
template <typename C> __device__ __forceinline__ C cconj(C a) { return {a.x, -a.y}; }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { return {a.x * s, a.y * s}; }
// a * s with each product rounded on its own (never fused into a later add): the first FFT pass
// feeds values formed on the way in straight into the DFT's additions, and a product the code
// generator was free to contract there could be fused differently in the plain and the batched
// instantiation of a kernel, which must agree bit for bit
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
template <typename C, typename T> __device__ __forceinline__ C cscale_rn(C a, T s) { return {mul_rn(a.x, s), mul_rn(a.y, s)}; }
// multiply by s*i
template <typename C> __device__ __forceinline__ C cmuli(C a, int s) { return s > 0 ? C{-a.y, a.x} : C{a.y, -a.x}; }

// In-place DFT of length R on v (sign s = -1 forward, +1 inverse).
template <typename C, typename T, int R>
__device__ __forceinline__ void dft(C* v, int s) {
  if constexpr (R == 2) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
  } else if constexpr (R == 3) {
    const T h = T(0.86602540378443864676);
    C t = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    C m = csub(v[0], cscale(t, T(0.5)));
    C r = cmuli(cscale(d, h), s);
    v[0] = cadd(v[0], t); v[1] = cadd(m, r); v[2] = csub(m, r);
  } else if constexpr (R == 4) {
    C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    C t2 = cadd(v[1], v[3]), t3 = cmuli(csub(v[1], v[3]), s);
    v[0] = cadd(t0, t2); v[2] = csub(t0, t2); v[1] = cadd(t1, t3); v[3] = csub(t1, t3);
  } else if constexpr (R == 8) {
    C e[4] = {v[0], v[2], v[4], v[6]}, o[4] = {v[1], v[3], v[5], v[7]};
    dft<C, T, 4>(e, s);
    dft<C, T, 4>(o, s);
    const T h = T(0.70710678118654752440);
    // twiddles e^{s 2 pi i k / 8}, k = 0..3
    C w1 = {h, T(s) * h}, w3 = {-h, T(s) * h};
    C o1 = cmul(o[1], w1), o2 = cmuli(o[2], s), o3 = cmul(o[3], w3);
    v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
    v[1] = cadd(e[1], o1);   v[5] = csub(e[1], o1);
    v[2] = cadd(e[2], o2);   v[6] = csub(e[2], o2);
    v[3] = cadd(e[3], o3);   v[7] = csub(e[3], o3);
  }
}

// Division by a divisor that is fixed for a whole loop: a shift and a mask when it is a power of
// two, else a float reciprocal with one correction step (exact for 0 <= x < 2^22; larger x divide).
struct IDiv {
  int d, sh;
  float inv;
  bool p2;
  // built once per thread and pass, for a handful of elements: the shift from a count of leading
  // zeros, the reciprocal (a division) only for divisors that need it
  __device__ __forceinline__ explicit IDiv(int d_) : d(d_), sh(0), inv(0.0f), p2((d_ & (d_ - 1)) == 0) {
#ifdef __CUDA_ARCH__
    if (p2) sh = 31 - __clz(d_);
    else inv = 1.0f / (float)d_;
#endif
  }
  __device__ __forceinline__ int div(int x) const {
    if (p2) return x >> sh;
    if (x >= (1 << 22)) return x / d;
    int q = __float2int_rz((float)x * inv);
    const int r = x - q * d;
    if (r >= d) ++q;
    else if (r < 0) --q;
    return q;
  }
  __device__ __forceinline__ int mod(int x) const { return p2 ? (x & (d - 1)) : x - div(x) * d; }
};

// Shared-memory layout of the FFT buffers: one padding element after every 128 bytes of data.
// A Stockham pass writes element j*R + r from the thread of butterfly j, a stride of R elements
// across the threads of a warp; unpadded, the first pass of a radix-8 x line puts a half-warp's
// sixteen 8-byte stores on two bank pairs (8-way conflict).  Padded, they fall on sixteen.
template <typename C> __host__ __device__ constexpr int spad_shift() { return sizeof(C) == 8 ? 4 : 3; }
template <typename C> __device__ __forceinline__ int spad(int i) { return i + (i >> spad_shift<C>()); }
// elements a buffer of n padded elements spans
template <typename C> __host__ __device__ constexpr size_t spad_size(size_t n) { return n + (n >> spad_shift<C>()); }

// One Stockham pass of radix R over `nlines` lines of length N: ld(l, e) supplies element e of
// line l, st(l, e, v) takes output element e of line l; twstep = N / (Ns R).  The twiddle table
// holds e^{-2 pi i t / (N*tws)} for t < N*tws (tws = stride into it).  A thread's R loads are issued
// together, before any of its stores.
template <typename C, typename T, int R, class Ld, class St>
__device__ __forceinline__ void stockham_pass(const Ld& ld, const St& st, int N, int Ns, int twstep, int nlines,
                                              const C* tw, int tws, int s, bool line_fast) {
  const int nb = N / R;
  const int total = nlines * nb;
  const IDiv dl(line_fast ? nlines : nb), dns(Ns);
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    int l, j;
    if (line_fast) { j = dl.div(idx); l = idx - j * nlines; }
    else { l = dl.div(idx); j = idx - l * nb; }
    C v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = ld(l, j + r * nb);
    const int jq = dns.div(j), k = j - jq * Ns;
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const int t = r * k * twstep;           // < N: k < Ns, r < R, twstep = N / (Ns R)
        C w = tw[t * tws];
        if (s > 0) w.y = -w.y;
        v[r] = cmul(v[r], w);
      }
    }
    dft<C, T, R>(v, s);
    const int base = jq * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) st(l, base + r * Ns, v[r]);
  }
}

// A pass whose input and output are each either the transform's own (ld / st: global memory or a
// computed value) or a padded shared buffer (element e of line l at spad(l*sl + e*se)).
template <typename C, typename T, int R, class Ld, class St>
__device__ __forceinline__ void stockham_pass_at(bool first, bool last, const Ld& ld, const St& st, const C* src,
                                                 C* dst, int sl, int se, int N, int Ns, int twstep, int nlines,
                                                 const C* tw, int tws, int s, bool line_fast, unsigned* oob) {
#if OCN_BOUNDS_CHECK
  const int cap = (int)spad_size<C>((size_t)nlines * N);   // elements of each shared buffer in use
#endif
  auto sld = [&](int l, int e) -> C { return src[OCN_CHK(spad<C>(l * sl + e * se), cap, oob, kOobFftShared)]; };
  auto sst = [&](int l, int e, C v) { dst[OCN_CHK(spad<C>(l * sl + e * se), cap, oob, kOobFftShared)] = v; };
  if (first && last) stockham_pass<C, T, R>(ld, st, N, Ns, twstep, nlines, tw, tws, s, line_fast);
  else if (first) stockham_pass<C, T, R>(ld, sst, N, Ns, twstep, nlines, tw, tws, s, line_fast);
  else if (last) stockham_pass<C, T, R>(sld, st, N, Ns, twstep, nlines, tw, tws, s, line_fast);
  else stockham_pass<C, T, R>(sld, sst, N, Ns, twstep, nlines, tw, tws, s, line_fast);
}

// Full FFT of `nlines` lines.  The first pass reads its input through ld(l, e) and the last pass
// writes its output through st(l, e, v), straight from and to global memory (or values computed
// on the way in), so only the passes in between go through shared memory: pass p writes buffer a
// for even p and b for odd p.  A one-pass transform touches no shared memory.  The last pass
// writes into the buffer the last pass of a transform through shared memory would use,
// (npass - 1) even ? a : b, when st stores there.
template <typename C, typename T, class Ld, class St>
__device__ __forceinline__ void block_fft(C* a, C* b, const FftPlan& plan, int nlines, int sl, int se, const C* tw,
                                          int tws, int s, bool line_fast, const Ld& ld, const St& st,
                                          unsigned* oob = nullptr) {
  int Ns = 1;
  int rem = plan.n;                      // N / Ns
  const int np = plan.npass;
  for (int p = 0; p < np; ++p) {
    const int R = plan.radix[p];
    const bool first = (p == 0), last = (p == np - 1);
    const C* src = (p & 1) ? a : b;      // written by pass p - 1
    C* dst = (p & 1) ? b : a;
    switch (R) {                         // rem / R = N / (Ns R), the pass's twiddle step
      case 8: rem /= 8; stockham_pass_at<C, T, 8>(first, last, ld, st, src, dst, sl, se, plan.n, Ns, rem, nlines, tw, tws, s, line_fast, oob); break;
      case 4: rem /= 4; stockham_pass_at<C, T, 4>(first, last, ld, st, src, dst, sl, se, plan.n, Ns, rem, nlines, tw, tws, s, line_fast, oob); break;
      case 3: rem /= 3; stockham_pass_at<C, T, 3>(first, last, ld, st, src, dst, sl, se, plan.n, Ns, rem, nlines, tw, tws, s, line_fast, oob); break;
      default: rem /= 2; stockham_pass_at<C, T, 2>(first, last, ld, st, src, dst, sl, se, plan.n, Ns, rem, nlines, tw, tws, s, line_fast, oob); break;
    }
    if (!last) __syncthreads();
    Ns *= R;
  }
}

// ---------------------------------------------------------------------------
// divergence + real FFT along x.  Each block handles LR consecutive rows.  The divergence goes to
// shared memory first, two elements per thread and trip with their loads issued together (taking
// it inside the first pass instead holds the six loads of each of a butterfly's eight elements at
// once: 64 registers and fewer blocks per SM, measured slower).
template <typename T>
__device__ __forceinline__ void div_fftx_body(const PoissonArgs<T>& a, int LR, const uint3 bid) {
  typedef typename CT<T>::type C;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* A = reinterpret_cast<C*>(sm_raw);
  const int M = a.Mx, Nx = a.Nx, Ny = a.Ny, Nz = a.Nz;
  C* B = A + spad_size<C>((size_t)LR * M);
  const size_t plane = (size_t)Nx * Ny;
  const int row0 = bid.x * LR;
  const int nrows = min(LR, Ny * Nz - row0);
  const IDiv dM(M), dNy(Ny);
  // pairs of cells as 2-vectors when the fields are aligned to them (the no-allocation projection
  // takes the caller's arrays)
  const bool pairs = ((reinterpret_cast<uintptr_t>(a.u) | reinterpret_cast<uintptr_t>(a.v) |
                       reinterpret_cast<uintptr_t>(a.w)) & (2 * sizeof(T) - 1)) == 0;
  // element n of line l: div(u)/dt at cells 2n and 2n+1 of row row0 + l (index of the second
  // element of a trip clamped into range; a clamped duplicate is not stored)
  const int ne = nrows * M;
  for (int b0 = threadIdx.x; b0 < ne; b0 += 2 * blockDim.x) {
    C out[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int idx = min(b0 + u * (int)blockDim.x, ne - 1);
      const int l = dM.div(idx), n = idx - l * M;
      const int row = row0 + l;
      const int k = dNy.div(row), j = row - k * Ny;
      const int jp = (j + 1 == Ny) ? 0 : j + 1;
      const T rdz = __ldg(a.rdzc + k);
      T val[2];
      const size_t o = OCN_CHK((size_t)k * plane + (size_t)j * Nx, (size_t)Nz * plane, a.oob, kOobFftGlobal);
      if (pairs) {                        // cells 2n, 2n+1 as one vector per field and level
        const C u01 = *reinterpret_cast<const C*>(a.u + o + 2 * n);
        const T u2 = a.u[o + (2 * n + 2 == Nx ? 0 : 2 * n + 2)];
        const C vj = *reinterpret_cast<const C*>(a.v + o + 2 * n);
        const C vp = *reinterpret_cast<const C*>(a.v + (size_t)k * plane + (size_t)jp * Nx + 2 * n);
        const C wk = *reinterpret_cast<const C*>(a.w + o + 2 * n);
        const C wt = *reinterpret_cast<const C*>(a.w + o + plane + 2 * n);
        val[0] = ((u01.y - u01.x) * a.rdx + (vp.x - vj.x) * a.rdy + (wt.x - wk.x) * rdz) * a.inv_dt;
        val[1] = ((u2 - u01.y) * a.rdx + (vp.y - vj.y) * a.rdy + (wt.y - wk.y) * rdz) * a.inv_dt;
      } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int i = 2 * n + h;
          const int ip = (i + 1 == Nx) ? 0 : i + 1;
          const T div = (a.u[o + ip] - a.u[o + i]) * a.rdx + (a.v[(size_t)k * plane + (size_t)jp * Nx + i] - a.v[o + i]) * a.rdy +
                        (a.w[o + plane + i] - a.w[o + i]) * rdz;
          val[h] = div * a.inv_dt;
        }
      }
      out[u] = C{val[0], val[1]};
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int idx = b0 + u * (int)blockDim.x;
      if (idx < ne) A[spad<C>(idx)] = out[u];       // idx = l * M + n
    }
  }
  __syncthreads();
  // the transform reads A in its first pass, so its passes write B first (block_fft(B, A, ..)),
  // and its output stays in shared memory for the split
  auto ld = [&](int l, int e) -> C { return A[spad<C>(l * M + e)]; };
  C* Z = ((a.px.npass - 1) & 1) ? A : B;
  auto st = [&](int l, int e, C v) { Z[spad<C>(l * M + e)] = v; };
  block_fft<C, T>(B, A, a.px, nrows, M, 1, reinterpret_cast<const C*>(a.twx), 2, -1, false, ld, st, a.oob);
  __syncthreads();
  // split: X[kx] = E + W^kx O, E = (Z[kx] + conj Z[M-kx])/2, O = (Z[kx] - conj Z[M-kx])/(2i)
  const int S = M + 1;
  const IDiv dS(S);
  for (int idx = threadIdx.x; idx < nrows * S; idx += blockDim.x) {
    const int l = dS.div(idx), kx = idx - l * S;          // kx = 0 .. M
    const C z1 = Z[spad<C>(l * M + (kx == M ? 0 : kx))];
    const C z2 = cconj(Z[spad<C>(l * M + (kx == 0 ? 0 : M - kx))]);
    const C E = cscale(cadd(z1, z2), T(0.5));
    const C D = cscale(csub(z1, z2), T(0.5));
    const C O = {D.y, -D.x};                   // D / i
    const C w = reinterpret_cast<const C*>(a.twx)[kx];    // kx <= M < Nx
    const C X = cadd(E, cmul(w, O));
    const int row = row0 + l;
    reinterpret_cast<C*>(a.spec)[OCN_CHK((size_t)row * a.Sp + kx, (size_t)Ny * Nz * a.Sp, a.oob, kOobFftGlobal)] = X;
  }
}

// complex-to-real inverse FFT along x -> p (scaled by a.scale).  The first pass forms its
// elements from the half spectrum; the last pass writes p.
template <typename T>
__device__ __forceinline__ void ifftx_body(const PoissonArgs<T>& a, int LR, const uint3 bid) {
  typedef typename CT<T>::type C;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* A = reinterpret_cast<C*>(sm_raw);
  const int M = a.Mx, Nx = a.Nx, Ny = a.Ny, Nz = a.Nz;
  C* B = A + spad_size<C>((size_t)LR * M);
  const int row0 = bid.x * LR;
  const int nrows = min(LR, Ny * Nz - row0);
  const C* spec = reinterpret_cast<const C*>(a.spec);
  const C* tw = reinterpret_cast<const C*>(a.twx);
  // element kx of line l: Z_kx = E + i e^{+2 pi i kx / Nx} O from X[kx] and conj X[M - kx]
  auto ld = [&](int l, int kx) -> C {
    const size_t ro = (size_t)(row0 + l) * a.Sp;
    [[maybe_unused]] const size_t nspec = (size_t)Ny * Nz * a.Sp;
    const C x1 = spec[OCN_CHK(ro + kx, nspec, a.oob, kOobFftGlobal)];
    const C x2 = cconj(spec[OCN_CHK(ro + (M - kx), nspec, a.oob, kOobFftGlobal)]);
    const C E = cscale(cadd(x1, x2), T(0.5));
    C w = tw[kx];
    w.y = -w.y;                                 // e^{+2 pi i kx / Nx}
    const C O = cmul(cscale(csub(x1, x2), T(0.5)), w);
    return cscale_rn(cadd(E, cmuli(O, 1)), a.scale);
  };
  const bool pairs = (reinterpret_cast<uintptr_t>(a.p) & (2 * sizeof(T) - 1)) == 0;   // p as 2-vectors
  // output element n of line l: p at cells 2n and 2n+1 of row row0 + l
  auto st = [&](int l, int n, C v) {
    const size_t o = OCN_CHK((size_t)(row0 + l) * Nx + 2 * n, (size_t)Nx * Ny * Nz - 1, a.oob, kOobFftGlobal);
    if (pairs) {
      *reinterpret_cast<C*>(a.p + o) = v;
    } else {
      a.p[o] = v.x;
      a.p[o + 1] = v.y;
    }
  };
  block_fft<C, T>(A, B, a.px, nrows, M, 1, tw, 2, +1, false, ld, st, a.oob);
}

// FFT along y of a tile of CW kx-columns in one z-plane, in place: the first pass reads the
// spectrum, the last pass writes it back (columns past the spectrum's edge are neither read nor
// written).  The Ny twiddles are staged in shared memory after the two data buffers; the first
// pass uses none (N_s = 1), and the barrier after it publishes them to the others.
template <typename T>
__device__ __forceinline__ void fft_y_body(const PoissonArgs<T>& a, int CW, int sign, const uint3 bid) {
  typedef typename CT<T>::type C;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* A = reinterpret_cast<C*>(sm_raw);
  const int Ny = a.Ny, S = a.Mx + 1, Sp = a.Sp;
  C* B = A + spad_size<C>((size_t)Ny * CW);
  C* sTw = B + spad_size<C>((size_t)Ny * CW);
  const int kx0 = bid.x * CW, k = bid.y;
  const int ncol = min(CW, S - kx0);
  C* spec = reinterpret_cast<C*>(a.spec) + (size_t)k * Ny * Sp;
  const C* twy = reinterpret_cast<const C*>(a.twy);
  for (int t = threadIdx.x; t < Ny; t += blockDim.x) sTw[t] = twy[t];
  [[maybe_unused]] const size_t nlev = (size_t)Ny * Sp;
  auto ld = [&](int l, int e) -> C {
    return (l < ncol) ? spec[OCN_CHK((size_t)e * Sp + kx0 + l, nlev, a.oob, kOobFftGlobal)] : C{T(0), T(0)};
  };
  auto st = [&](int l, int e, C v) { if (l < ncol) spec[OCN_CHK((size_t)e * Sp + kx0 + l, nlev, a.oob, kOobFftGlobal)] = v; };
  block_fft<C, T>(A, B, a.py, CW, 1, CW, sTw, 1, sign, true, ld, st, a.oob);
}

// Thomas algorithm per horizontal wavenumber.  a_k p_{k-1} + b_k p_k + c_k p_{k+1} = r_k,
// a_k = 1/(dzc_k dzf_k), c_k = 1/(dzc_k dzf_{k+1}) (zero at the walls: Neumann),
// b_k = -(a_k + c_k) + lambda_x + lambda_y; the (0,0) column's first row is p_0 = 0 (gauge).
// The coefficients depend only on the grid, so the elimination is factored once
// (k_tridiag_factor: c'_k and 1/(b_k - a_k c'_{k-1}) in precision P, stored in T) and each solve
// is two sweeps of multiply-adds (k_tridiag_solve), levels moved in batches of kTriChunk so that
// their loads are issued together.  k_tridiag factors and solves in one pass (for callers
// without the factor arrays).
template <typename T, typename P>
__device__ __forceinline__ void tri_coeffs(const PoissonArgs<T>& a, int k, int Nz, P lam, bool gauge, P& ak, P& bk,
                                           P& ck) {
  const P rz = (P)__ldg(a.rdzc + k);
  ak = (k > 0) ? rz * (P)__ldg(a.rdzf + k) : P(0);
  ck = (k < Nz - 1) ? rz * (P)__ldg(a.rdzf + k + 1) : P(0);
  bk = -(ak + ck) + lam;
  if (gauge && k == 0) { ak = P(0); bk = P(1); ck = P(0); }
}

template <typename T, typename P>
__device__ __forceinline__ void tridiag_body(const PoissonArgs<T>& a, const uint3 bid) {
  typedef typename CT<T>::type C;
  const int S = a.Mx + 1, Ny = a.Ny, Nz = a.Nz;
  const int o_ = bid.x * blockDim.x + threadIdx.x;   // column ky * S + kx
  if (o_ >= S * Ny) return;
  const int ky = o_ / S, kx = o_ - ky * S;
  const size_t pl = (size_t)Ny * a.Sp;
  C* x = reinterpret_cast<C*>(a.spec) + (size_t)ky * a.Sp + kx;
  T* cp = a.cpiv + (size_t)ky * a.Sp + kx;
  const P lam = (P)__ldg(a.lamx + kx) + (P)__ldg(a.lamy + ky);
  const bool gauge = (kx == 0 && ky == 0);
  P cprev = P(0);
  C dprev = {T(0), T(0)};
  for (int k = 0; k < Nz; ++k) {
    P ak, bk, ck;
    tri_coeffs<T, P>(a, k, Nz, lam, gauge, ak, bk, ck);
    C r = x[(size_t)k * pl];
    if (gauge && k == 0) r = C{T(0), T(0)};
    const P inv = P(1) / (bk - ak * cprev);
    cprev = ck * inv;
    const T ti = (T)inv, ta = (T)ak;
    C d = {(r.x - ta * dprev.x) * ti, (r.y - ta * dprev.y) * ti};
    x[(size_t)k * pl] = d;
    cp[(size_t)k * pl] = (T)cprev;
    dprev = d;
  }
  C pn = dprev;
  for (int k = Nz - 2; k >= 0; --k) {
    const T c = cp[(size_t)k * pl];
    C d = x[(size_t)k * pl];
    d.x -= c * pn.x;
    d.y -= c * pn.y;
    x[(size_t)k * pl] = d;
    pn = d;
  }
}

template <typename T, typename P>
__global__ void __launch_bounds__(256) k_tridiag_factor(const PoissonArgs<T> a) {
  const int S = a.Mx + 1, Ny = a.Ny, Nz = a.Nz;
  const int o_ = blockIdx.x * blockDim.x + threadIdx.x;   // column ky * S + kx
  if (o_ >= S * Ny) return;
  const int ky = o_ / S, kx = o_ - ky * S;
  const size_t pl = (size_t)Ny * a.Sp, o = (size_t)ky * a.Sp + kx;
  const P lam = (P)__ldg(a.lamx + kx) + (P)__ldg(a.lamy + ky);
  const bool gauge = (kx == 0 && ky == 0);
  P cprev = P(0);
  for (int k = 0; k < Nz; ++k) {
    P ak, bk, ck;
    tri_coeffs<T, P>(a, k, Nz, lam, gauge, ak, bk, ck);
    const P inv = P(1) / (bk - ak * cprev);
    cprev = ck * inv;
    a.pinv[(size_t)k * pl + o] = (T)inv;
    a.cpiv[(size_t)k * pl + o] = (T)cprev;
  }
}

constexpr int kTriChunk = 8;

template <typename T>
__device__ __forceinline__ void tridiag_solve_body(const PoissonArgs<T>& a, const uint3 bid) {
  typedef typename CT<T>::type C;
  const int S = a.Mx + 1, Ny = a.Ny, Nz = a.Nz;
  const int o_ = bid.x * blockDim.x + threadIdx.x;   // column ky * S + kx
  if (o_ >= S * Ny) return;
  const int ky = o_ / S, kx = o_ - ky * S;
  const size_t pl = (size_t)Ny * a.Sp, o = (size_t)ky * a.Sp + kx;
#if OCN_BOUNDS_CHECK
  // the column's unknowns and factors, levels 0 .. Nz-1, inside the spectrum
  (void)OCN_CHK(o + (size_t)(Nz - 1) * pl, pl * (size_t)Nz, a.oob, kOobTridiag);
#endif
  C* x = reinterpret_cast<C*>(a.spec) + o;
  const T* cp = a.cpiv + o;
  const T* pinv = a.pinv + o;
  const bool gauge = (kx == 0 && ky == 0);
  C dprev = {T(0), T(0)};
  for (int k0 = 0; k0 < Nz; k0 += kTriChunk) {
    C r[kTriChunk];
    T iv[kTriChunk];
#pragma unroll
    for (int u = 0; u < kTriChunk; ++u) {
      const int k = k0 + u;
      r[u] = (k < Nz) ? x[(size_t)k * pl] : C{T(0), T(0)};
      iv[u] = (k < Nz) ? __ldg(pinv + (size_t)k * pl) : T(0);
    }
#pragma unroll
    for (int u = 0; u < kTriChunk; ++u) {
      const int k = k0 + u;
      if (k < Nz) {
        const T ta = (k > 0) ? __ldg(a.rdzc + k) * __ldg(a.rdzf + k) : T(0);
        C rr = r[u];
        if (gauge && k == 0) rr = C{T(0), T(0)};
        dprev = C{(rr.x - ta * dprev.x) * iv[u], (rr.y - ta * dprev.y) * iv[u]};
        r[u] = dprev;
      }
    }
#pragma unroll
    for (int u = 0; u < kTriChunk; ++u)
      if (k0 + u < Nz) x[(size_t)(k0 + u) * pl] = r[u];
  }
  C pn = dprev;
  for (int k1 = Nz - 2; k1 >= 0; k1 -= kTriChunk) {
    C d[kTriChunk];
    T c[kTriChunk];
#pragma unroll
    for (int u = 0; u < kTriChunk; ++u) {
      const int k = k1 - u;
      d[u] = (k >= 0) ? x[(size_t)k * pl] : C{T(0), T(0)};
      c[u] = (k >= 0) ? __ldg(cp + (size_t)k * pl) : T(0);
    }
#pragma unroll
    for (int u = 0; u < kTriChunk; ++u) {
      if (k1 - u >= 0) {
        d[u].x -= c[u] * pn.x;
        d[u].y -= c[u] * pn.y;
        pn = d[u];
      }
    }
#pragma unroll
    for (int u = 0; u < kTriChunk; ++u)
      if (k1 - u >= 0) x[(size_t)(k1 - u) * pl] = d[u];
  }
}

// zero volume mean of the (kx,ky) = (0,0) column (one warp)
template <typename T>
__device__ __forceinline__ void gauge_body(const PoissonArgs<T>& a) {
  typedef typename CT<T>::type C;
  const size_t pl = (size_t)a.Ny * a.Sp;
  C* x = reinterpret_cast<C*>(a.spec);
  double sr = 0.0, si = 0.0;
  for (int k = threadIdx.x; k < a.Nz; k += 32) {
    const double dz = (double)a.dzc[k];
    sr += dz * (double)x[(size_t)k * pl].x;
    si += dz * (double)x[(size_t)k * pl].y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  const T mr = (T)(sr / (double)a.Htot), mi = (T)(si / (double)a.Htot);
  for (int k = threadIdx.x; k < a.Nz; k += 32) {
    C v = x[(size_t)k * pl];
    v.x -= mr;
    v.y -= mi;
    x[(size_t)k * pl] = v;
  }
}

// u = u~ - dt grad p (walls untouched)
template <typename T>
__device__ __forceinline__ void correct_body(const PoissonArgs<T>& a, const uint3 bid) {
  const int Nx = a.Nx, Ny = a.Ny;
  const int c = bid.x * blockDim.x + threadIdx.x;   // j * Nx + i (narrow grids fill the blocks)
  const int k = bid.y;
  if (c >= Nx * Ny) return;
  const int j = c / Nx, i = c - j * Nx;
  const size_t plane = (size_t)Nx * Ny;
  const size_t id = (size_t)k * plane + (size_t)j * Nx + i;
  const int im = (i == 0) ? Nx - 1 : i - 1;
  const int jm = (j == 0) ? Ny - 1 : j - 1;
  const T pc = a.p[id];
  a.u[id] -= a.dt * (pc - a.p[(size_t)k * plane + (size_t)j * Nx + im]) * a.rdx;
  a.v[id] -= a.dt * (pc - a.p[(size_t)k * plane + (size_t)jm * Nx + i]) * a.rdy;
  if (k >= 1) a.w[id] -= a.dt * (pc - a.p[id - plane]) * __ldg(a.rdzf + k);
}

// The same correction for four consecutive cells of a row per thread (FP32, Nx a multiple of 4):
// 16-byte loads and stores, the same arithmetic per cell.
__device__ __forceinline__ void correct4_body(const PoissonArgs<float>& a, const uint3 bid) {
  const int Nx = a.Nx, Ny = a.Ny;
  const int c = (bid.x * blockDim.x + threadIdx.x) * 4;   // j * Nx + i, i a multiple of 4
  const int k = bid.y;
  if (c >= Nx * Ny) return;
  const int j = c / Nx, i = c - j * Nx;
  const size_t plane = (size_t)Nx * Ny;
  const size_t id = (size_t)k * plane + (size_t)j * Nx + i;
  const int jm = (j == 0) ? Ny - 1 : j - 1;
  const float4 pc = *reinterpret_cast<const float4*>(a.p + id);
  const float pw = a.p[(size_t)k * plane + (size_t)j * Nx + (i == 0 ? Nx - 1 : i - 1)];
  const float4 ps = *reinterpret_cast<const float4*>(a.p + (size_t)k * plane + (size_t)jm * Nx + i);
  float4 u = *reinterpret_cast<const float4*>(a.u + id);
  float4 v = *reinterpret_cast<const float4*>(a.v + id);
  const float dt = a.dt, rdx = a.rdx, rdy = a.rdy;
  u.x -= dt * (pc.x - pw) * rdx;
  u.y -= dt * (pc.y - pc.x) * rdx;
  u.z -= dt * (pc.z - pc.y) * rdx;
  u.w -= dt * (pc.w - pc.z) * rdx;
  v.x -= dt * (pc.x - ps.x) * rdy;
  v.y -= dt * (pc.y - ps.y) * rdy;
  v.z -= dt * (pc.z - ps.z) * rdy;
  v.w -= dt * (pc.w - ps.w) * rdy;
  *reinterpret_cast<float4*>(a.u + id) = u;
  *reinterpret_cast<float4*>(a.v + id) = v;
  if (k >= 1) {
    const float4 pb = *reinterpret_cast<const float4*>(a.p + id - plane);
    const float rz = __ldg(a.rdzf + k);
    float4 w = *reinterpret_cast<const float4*>(a.w + id);
    w.x -= dt * (pc.x - pb.x) * rz;
    w.y -= dt * (pc.y - pb.y) * rz;
    w.z -= dt * (pc.z - pb.z) * rz;
    w.w -= dt * (pc.w - pb.w) * rz;
    *reinterpret_cast<float4*>(a.w + id) = w;
  }
}

// Plain kernels and their batched forms (k_batched over the *K bodies).
template <typename T>
struct PoissonLaunch {            // the projection's arguments and the launch integers of one kernel
  PoissonArgs<T> a;
  int i0, i1;
};
template <typename T> struct DivFftxK {
  typedef PoissonLaunch<T> Payload;
  static constexpr int kThreads = 256, kMinBlocks = 1;
  static __device__ __forceinline__ void run(const Payload& p, uint3 bid, uint3) { div_fftx_body<T>(p.a, p.i0, bid); }
};
template <typename T> struct IfftxK {
  typedef PoissonLaunch<T> Payload;
  static constexpr int kThreads = 256, kMinBlocks = 1;
  static __device__ __forceinline__ void run(const Payload& p, uint3 bid, uint3) { ifftx_body<T>(p.a, p.i0, bid); }
};
template <typename T> struct FftYK {
  typedef PoissonLaunch<T> Payload;
  static constexpr int kThreads = 256, kMinBlocks = 1;
  static __device__ __forceinline__ void run(const Payload& p, uint3 bid, uint3) { fft_y_body<T>(p.a, p.i0, p.i1, bid); }
};
template <typename T, typename P> struct TridiagK {
  typedef PoissonArgs<T> Payload;
  static constexpr int kThreads = 256, kMinBlocks = 1;
  static __device__ __forceinline__ void run(const Payload& a, uint3 bid, uint3) { tridiag_body<T, P>(a, bid); }
};
template <typename T> struct TridiagSolveK {
  typedef PoissonArgs<T> Payload;
  static constexpr int kThreads = 256, kMinBlocks = 1;
  static __device__ __forceinline__ void run(const Payload& a, uint3 bid, uint3) { tridiag_solve_body<T>(a, bid); }
};
template <typename T> struct GaugeK {
  typedef PoissonArgs<T> Payload;
  static constexpr int kThreads = 32, kMinBlocks = 1;
  static __device__ __forceinline__ void run(const Payload& a, uint3, uint3) { gauge_body<T>(a); }
};
template <typename T> struct CorrectK {
  typedef PoissonArgs<T> Payload;
  static constexpr int kThreads = 256, kMinBlocks = 1;
  static __device__ __forceinline__ void run(const Payload& a, uint3 bid, uint3) { correct_body<T>(a, bid); }
};
struct Correct4K {
  typedef PoissonArgs<float> Payload;
  static constexpr int kThreads = 256, kMinBlocks = 1;
  static __device__ __forceinline__ void run(const Payload& a, uint3 bid, uint3) { correct4_body(a, bid); }
};

template <typename T>
__global__ void __launch_bounds__(256) k_div_fftx(const PoissonArgs<T> a, int LR) { div_fftx_body<T>(a, LR, blockIdx); }
template <typename T>
__global__ void __launch_bounds__(256) k_ifftx(const PoissonArgs<T> a, int LR) { ifftx_body<T>(a, LR, blockIdx); }
template <typename T>
__global__ void __launch_bounds__(256) k_fft_y(const PoissonArgs<T> a, int CW, int sign) {
  fft_y_body<T>(a, CW, sign, blockIdx);
}
template <typename T, typename P>
__global__ void __launch_bounds__(256) k_tridiag(const PoissonArgs<T> a) { tridiag_body<T, P>(a, blockIdx); }
template <typename T>
__global__ void __launch_bounds__(256) k_tridiag_solve(const PoissonArgs<T> a) { tridiag_solve_body<T>(a, blockIdx); }
template <typename T>
__global__ void k_gauge(const PoissonArgs<T> a) { gauge_body<T>(a); }
template <typename T>
__global__ void __launch_bounds__(256) k_correct(const PoissonArgs<T> a) { correct_body<T>(a, blockIdx); }
__global__ void __launch_bounds__(256) k_correct4(const PoissonArgs<float> a) { correct4_body(a, blockIdx); }

template <typename T>
static PoissonLaunch<T> with_ints(const PoissonArgs<T>& a, int i0, int i1) {
  PoissonLaunch<T> p;
  memset(&p, 0, sizeof(p));
  p.a = a; p.i0 = i0; p.i1 = i1;
  return p;
}

static int rows_per_block(int M) { return M >= 2048 ? 1 : 2048 / M; }

template <typename T>
cudaError_t launch_projection(const PoissonArgs<T>& a, cudaStream_t s, int* nlaunch, const LaunchHook& hook) {
  typedef typename CT<T>::type C;
  cudaError_t e;
  int n = 0;
  const int M = a.Mx;
  const int LR = rows_per_block(M);
  const size_t smx = 2 * spad_size<C>((size_t)LR * M) * sizeof(C);
  const int rows = a.Ny * a.Nz;
  e = raise_smem_limit(k_div_fftx<T>, smx);
  if (e != cudaSuccess) return e;
  e = raise_smem_limit(k_ifftx<T>, smx);
  if (e != cudaSuccess) return e;
  const bool rec = active_recorder() != nullptr;
  hook.pre(OCN_K_DIV_FFTX);
  if (!record_launch<DivFftxK<T>>(with_ints(a, LR, 0), dim3((rows + LR - 1) / LR), dim3(256), smx, OCN_K_DIV_FFTX))
    k_div_fftx<T><<<(rows + LR - 1) / LR, 256, smx, s>>>(a, LR);
  hook.post(OCN_K_DIV_FFTX);
  ++n;
  // kx columns per block: four (32 bytes of each row in FP32, a whole sector), widened for short y
  // lines so that a block holds about 2048 (FP32) / 1024 (FP64) values, not beyond the spectrum
  int CW = 4;
  while (CW * a.Ny < (sizeof(T) == 4 ? 2048 : 1024) && CW < a.Mx + 1) CW *= 2;
  const size_t smy = (2 * spad_size<C>((size_t)a.Ny * CW) + a.Ny) * sizeof(C);
  e = raise_smem_limit(k_fft_y<T>, smy);
  if (e != cudaSuccess) return e;
  dim3 gy((a.Mx + 1 + CW - 1) / CW, a.Nz);
  hook.pre(OCN_K_FFT_Y);
  if (!record_launch<FftYK<T>>(with_ints(a, CW, -1), gy, dim3(256), smy, OCN_K_FFT_Y)) k_fft_y<T><<<gy, 256, smy, s>>>(a, CW, -1);
  hook.post(OCN_K_FFT_Y);
  ++n;
  dim3 gt(((a.Mx + 1) * a.Ny + 127) / 128);
  hook.pre(OCN_K_TRIDIAG);
  if (a.pinv) {
    if (!record_launch<TridiagSolveK<T>>(a, gt, dim3(128), 0, OCN_K_TRIDIAG)) k_tridiag_solve<T><<<gt, 128, 0, s>>>(a);
  } else if (a.fp64_pivots) {
    if (!record_launch<TridiagK<T, double>>(a, gt, dim3(128), 0, OCN_K_TRIDIAG)) k_tridiag<T, double><<<gt, 128, 0, s>>>(a);
  } else {
    if (!record_launch<TridiagK<T, T>>(a, gt, dim3(128), 0, OCN_K_TRIDIAG)) k_tridiag<T, T><<<gt, 128, 0, s>>>(a);
  }
  hook.post(OCN_K_TRIDIAG);
  ++n;
  hook.pre(OCN_K_GAUGE);
  if (!record_launch<GaugeK<T>>(a, dim3(1), dim3(32), 0, OCN_K_GAUGE)) k_gauge<T><<<1, 32, 0, s>>>(a);
  hook.post(OCN_K_GAUGE);
  ++n;
  hook.pre(OCN_K_FFT_Y);
  if (!record_launch<FftYK<T>>(with_ints(a, CW, +1), gy, dim3(256), smy, OCN_K_FFT_Y)) k_fft_y<T><<<gy, 256, smy, s>>>(a, CW, +1);
  hook.post(OCN_K_FFT_Y);
  ++n;
  hook.pre(OCN_K_IFFTX);
  if (!record_launch<IfftxK<T>>(with_ints(a, LR, 0), dim3((rows + LR - 1) / LR), dim3(256), smx, OCN_K_IFFTX))
    k_ifftx<T><<<(rows + LR - 1) / LR, 256, smx, s>>>(a, LR);
  hook.post(OCN_K_IFFTX);
  ++n;
  hook.pre(OCN_K_CORRECT);
  // 16-byte vectors need rows of a multiple of 4 cells and 16-byte aligned fields (a caller of the
  // no-allocation projection supplies its own)
  const bool vec4 = std::is_same<T, float>::value && a.Nx % 4 == 0 &&
                    ((reinterpret_cast<uintptr_t>(a.u) | reinterpret_cast<uintptr_t>(a.v) |
                      reinterpret_cast<uintptr_t>(a.w) | reinterpret_cast<uintptr_t>(a.p)) & 15) == 0;
  if constexpr (std::is_same<T, float>::value) {
    if (vec4) {
      dim3 gc4((a.Nx * a.Ny / 4 + 255) / 256, a.Nz);
      if (!record_launch<Correct4K>(a, gc4, dim3(256), 0, OCN_K_CORRECT)) k_correct4<<<gc4, 256, 0, s>>>(a);
    }
  }
  if (!vec4) {
    dim3 gc((a.Nx * a.Ny + 255) / 256, a.Nz);
    if (!record_launch<CorrectK<T>>(a, gc, dim3(256), 0, OCN_K_CORRECT)) k_correct<T><<<gc, 256, 0, s>>>(a);
  }
  hook.post(OCN_K_CORRECT);
  ++n;
  if (nlaunch) *nlaunch = n;
  return rec ? cudaSuccess : cudaGetLastError();
}

template <typename T>
cudaError_t launch_tridiag_factor(const PoissonArgs<T>& a, cudaStream_t s) {
  if (!a.pinv || !a.cpiv) return cudaErrorInvalidValue;
  dim3 gt(((a.Mx + 1) * a.Ny + 127) / 128);
  if (a.fp64_pivots) k_tridiag_factor<T, double><<<gt, 128, 0, s>>>(a);
  else k_tridiag_factor<T, T><<<gt, 128, 0, s>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_tridiag_factor<float>(const PoissonArgs<float>&, cudaStream_t);
template cudaError_t launch_tridiag_factor<double>(const PoissonArgs<double>&, cudaStream_t);

template cudaError_t launch_projection<float>(const PoissonArgs<float>&, cudaStream_t, int*, const LaunchHook&);
template cudaError_t launch_projection<double>(const PoissonArgs<double>&, cudaStream_t, int*, const LaunchHook&);

}  // namespace ocn
