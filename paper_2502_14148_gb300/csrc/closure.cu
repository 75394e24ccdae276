// Eddy diffusivities (Smagorinsky-Lilly, AMD) at cell centres.
#include <cuda_runtime.h>

#include <algorithm>

#include "batch.cuh"
#include "ocn_internal.cuh"

namespace ocn {

// Eddy diffusivities at cell centres (Sec. 3.1.1): Smagorinsky-Lilly and AMD.
// One thread per (i, j) column marching up in z: the values on face / level
// k+1 loaded for one level are reused as the k values of the next, so each cell
// costs about twenty loads (horizontal neighbours come through L1).  The march is
// bound by load latency and instruction issue together, so residency matters: in FP32,
// four 256-thread CTAs per SM (registers capped at 64) measured 1.5x faster than three;
// more CTAs spill.
// SMAG: compiled for Smagorinsky-Lilly (true) or AMD (false).
//
// Each level's new values come from HBM with nothing else in flight for that warp, so the
// march also asks L2 for the column's values kPrefetch levels ahead (prefetch.global.L2: no
// register, no wait); the loads of those levels then hit L2.  (Unrolling the march by two levels,
// so that both levels' loads are issued together, spills under the 64-register cap and measured
// slower.)
constexpr int kPrefetch = 3;
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <typename T, bool SMAG>
__device__ __forceinline__ void closure_body(const ClosureArgs<T>& a, const uint3 bid, const uint3 gdim) {
  const int i = bid.x * blockDim.x + threadIdx.x;
  const int j = bid.y * blockDim.y + threadIdx.y;
  const int Nx = a.Nx, Ny = a.Ny, Nz = a.Nz;
  if (i >= Nx || j >= Ny) return;
  const size_t plane = (size_t)Nx * Ny;
  const int ip = (i + 1 == Nx) ? 0 : i + 1, im = (i == 0) ? Nx - 1 : i - 1;
  const int jp = (j + 1 == Ny) ? 0 : j + 1, jm = (j == 0) ? Ny - 1 : j - 1;
  // column offsets inside a level, 32-bit (grids are created with Nx Ny < 2^31): the march keeps
  // one pointer per field to its current level, so a load adds a 32-bit offset to it instead of
  // forming a 64-bit level-plus-column index
  const int c00 = j * Nx + i, cp0 = j * Nx + ip, cm0 = j * Nx + im;
  const int c0p = jp * Nx + i, c0m = jm * Nx + i;
  const int cpp = jp * Nx + ip, cpm = jm * Nx + ip, cmp = jp * Nx + im;
  const T rdx = a.rdx, rdy = a.rdy;
  const bool ts = (a.eos == OCN_EOS_LINEAR_TS);
  const T* cr0 = a.cref[0];
  const T* cr1 = a.cref[1];
  auto cref = [&](int t, int kk) -> T { return a.cref[t] ? __ldg(a.cref[t] + kk) : T(0); };
  // b at (i, j) from the tracers of a level (pointers to it) and level kk's reference profiles
  auto buoy = [&](const T* c0, const T* c1, int kk) -> T {
    const T t0 = __ldg(c0 + c00) + (cr0 ? __ldg(cr0 + kk) : T(0));
    if (ts) return a.g_alpha * (t0 - a.T0) - a.g_beta * (__ldg(c1 + c00) + (cr1 ? __ldg(cr1 + kk) : T(0)) - a.S0);
    return t0;
  };
  // this CTA's chunk of levels [kb, ke) (block z); the march state is set up at kb from the level
  // below, so chunks are independent
  const int nch = gdim.z, per = (Nz + nch - 1) / nch;
  const int kb = bid.z * per, ke = min(Nz, kb + per);
  if (kb >= ke) return;
  // level-kb pointers (w: face kb); tracer pointers are only formed for the tracers a kernel reads
  const T* Uk = a.cur.u + (size_t)kb * plane;
  const T* Vk = a.cur.v + (size_t)kb * plane;
  const T* Wk = a.cur.w + (size_t)kb * plane;
  const T* C0k = SMAG ? a.cur.c[0] + (size_t)kb * plane : nullptr;
  const T* C1k = (SMAG && ts) ? a.cur.c[1] + (size_t)kb * plane : nullptr;
  // carried from level to level: u at (i|ip, j) and v at (i, j|jp) on the current level, w on face k,
  // the two lower-face z-derivatives, b below
  T u0 = __ldg(Uk + c00), u1 = __ldg(Uk + cp0);
  T v0 = __ldg(Vk + c00), v1 = __ldg(Vk + c0p);
  T w00 = __ldg(Wk + c00), wm0 = __ldg(Wk + cm0), wp0 = __ldg(Wk + cp0), w0m = __ldg(Wk + c0m), w0p = __ldg(Wk + c0p);
  T dudz_lo0 = T(0), dudz_lo1 = T(0), dvdz_lo0 = T(0), dvdz_lo1 = T(0);   // faces at k (walls: 0)
  if (kb > 0) {
    const T r = __ldg(a.rdzf + kb);
    dudz_lo0 = (u0 - __ldg(Uk - plane + c00)) * r;
    dudz_lo1 = (u1 - __ldg(Uk - plane + cp0)) * r;
    dvdz_lo0 = (v0 - __ldg(Vk - plane + c00)) * r;
    dvdz_lo1 = (v1 - __ldg(Vk - plane + c0p)) * r;
  }
  T b_prev = T(0), b_cur = T(0);
  if constexpr (SMAG) {
    if (kb > 0) b_prev = buoy(C0k - plane, ts ? C1k - plane : nullptr, kb - 1);
    b_cur = buoy(C0k, C1k, kb);
  }
  for (int k = kb; k < ke; ++k) {
    const T* U1 = Uk + plane;               // level k+1 (face k+1 for w)
    const T* V1 = Vk + plane;
    const T* W1 = Wk + plane;
    {
      // level (and face) k+1+kPrefetch, in bounds only
      const int kp = k + 1 + kPrefetch;
      const size_t ahead = (size_t)kPrefetch * plane;
      if (kp <= Nz) prefetch_l2(W1 + ahead + c00);
      if (kp < Nz) {
        prefetch_l2(U1 + ahead + c00);
        prefetch_l2(V1 + ahead + c00);
        if constexpr (SMAG) {
          prefetch_l2(C0k + plane + ahead + c00);
          if (ts) prefetch_l2(C1k + plane + ahead + c00);
        } else {
          for (int t = 0; t < a.nt; ++t) prefetch_l2(a.cur.c[t] + (size_t)kp * plane + c00);
        }
      }
    }
    const T rdzc = __ldg(a.rdzc + k);
    const T rdzf1 = (k + 1 < Nz) ? __ldg(a.rdzf + k + 1) : T(0);
    const T dz = __ldg(a.dzc + k);
    // next level (k+1) of the carried columns, and face k+1 of w
    T un0 = T(0), un1 = T(0), vn0 = T(0), vn1 = T(0);
    if (k + 1 < Nz) { un0 = __ldg(U1 + c00); un1 = __ldg(U1 + cp0); vn0 = __ldg(V1 + c00); vn1 = __ldg(V1 + c0p); }
    const T w01 = __ldg(W1 + c00), wm1 = __ldg(W1 + cm0), wp1 = __ldg(W1 + cp0);
    const T w0m1 = __ldg(W1 + c0m), w0p1 = __ldg(W1 + c0p);
    // horizontal neighbours on level k
    const T u_0m = __ldg(Uk + c0m), u_1m = __ldg(Uk + cpm), u_0p = __ldg(Uk + c0p), u_1p = __ldg(Uk + cpp);
    const T v_m0 = __ldg(Vk + cm0), v_p0 = __ldg(Vk + cp0), v_mp = __ldg(Vk + cmp), v_pp = __ldg(Vk + cpp);
    const T ux = (u1 - u0) * rdx;
    const T vy = (v1 - v0) * rdy;
    const T wz = (w01 - w00) * rdzc;
    // d u/dy at the four (f, f) edges around the centre, d v/dx likewise
    const T uy = T(0.25) * ((u0 - u_0m) + (u1 - u_1m) + (u_0p - u0) + (u_1p - u1)) * rdy;
    const T vx = T(0.25) * ((v0 - v_m0) + (v_p0 - v0) + (v1 - v_mp) + (v_pp - v1)) * rdx;
    // z-derivatives on face k+1 (walls: 0), averaged with face k
    const T dudz_hi0 = (k + 1 < Nz) ? (un0 - u0) * rdzf1 : T(0);
    const T dudz_hi1 = (k + 1 < Nz) ? (un1 - u1) * rdzf1 : T(0);
    const T dvdz_hi0 = (k + 1 < Nz) ? (vn0 - v0) * rdzf1 : T(0);
    const T dvdz_hi1 = (k + 1 < Nz) ? (vn1 - v1) * rdzf1 : T(0);
    const T uz = T(0.25) * (dudz_lo0 + dudz_lo1 + dudz_hi0 + dudz_hi1);
    const T vz = T(0.25) * (dvdz_lo0 + dvdz_lo1 + dvdz_hi0 + dvdz_hi1);
    const T wx = T(0.25) * ((w00 - wm0) + (wp0 - w00) + (w01 - wm1) + (wp1 - w01)) * rdx;
    const T wy = T(0.25) * ((w00 - w0m) + (w0p - w00) + (w01 - w0m1) + (w0p1 - w01)) * rdy;
    const size_t id = (size_t)k * plane + c00;
    if constexpr (SMAG) {
      const T b_next = (k + 1 < Nz) ? buoy(C0k + plane, ts ? C1k + plane : nullptr, k + 1) : T(0);
      const T S12 = T(0.5) * (uy + vx), S13 = T(0.5) * (uz + wx), S23 = T(0.5) * (vz + wy);
      const T SS = T(2) * (ux * ux + vy * vy + wz * wz + T(2) * (S12 * S12 + S13 * S13 + S23 * S23));
      T nu = T(0);
      if (SS > T(0)) {
        const T dbb = (k >= 1) ? (b_cur - b_prev) * __ldg(a.rdzf + k) : T(0);
        const T dbt = (k + 1 < Nz) ? (b_next - b_cur) * rdzf1 : T(0);
        const T N2 = T(0.5) * (dbb + dbt);
        const T Delta = cbrt(a.dx * a.dy * dz);
        const T CD = a.Cs * Delta;
        // (C_s Delta)^2 sqrt(SS) sqrt(max(1 - C_b N2 / (Pr SS), 0)), written for SS > 0 without the division
        const T e = SS - a.Cb * N2 * a.inv_Pr;
        nu = e > T(0) ? CD * CD * sqrt(e) : T(0);
      }
      a.nu[id] = nu;
      b_prev = b_cur;
      b_cur = b_next;
      C0k += plane;
      if (ts) C1k += plane;
    } else {  // AMD
      const T G[3][3] = {{ux, uy, uz}, {vx, vy, vz}, {wx, wy, wz}};
      const T D2[3] = {a.dx * a.dx, a.dy * a.dy, dz * dz};
      // num = sum_m D2_m g_m^T S g_m over the columns g_m = G[.][m]; with S the symmetric part of G,
      // g^T S g = g^T G g, so each term is one matrix-vector product and a dot product
      T num = T(0), den = T(0);
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        T h = T(0);
#pragma unroll
        for (int p = 0; p < 3; ++p) h += G[p][m] * (G[p][0] * G[0][m] + G[p][1] * G[1][m] + G[p][2] * G[2][m]);
        num += D2[m] * h;
      }
#pragma unroll
      for (int p = 0; p < 3; ++p)
#pragma unroll
        for (int q = 0; q < 3; ++q) den += G[p][q] * G[p][q];
      T nu = (den > T(0)) ? -a.C_amd * num / den : T(0);
      a.nu[id] = nu > T(0) ? nu : T(0);
      for (int t = 0; t < a.nt; ++t) {
        const T* c = a.cur.c[t] + (size_t)k * plane;      // level k of tracer t
        const T c0 = __ldg(c + c00);
        T dc[3];
        dc[0] = T(0.5) * ((c0 - __ldg(c + cm0)) + (__ldg(c + cp0) - c0)) * rdx;
        dc[1] = T(0.5) * ((c0 - __ldg(c + c0m)) + (__ldg(c + c0p) - c0)) * rdy;
        const T dcb = (k >= 1) ? ((c0 - __ldg(c - plane + c00)) + (cref(t, k) - cref(t, k - 1))) * __ldg(a.rdzf + k) : T(0);
        const T dct = (k + 1 < Nz) ? ((__ldg(c + plane + c00) - c0) + (cref(t, k + 1) - cref(t, k))) * rdzf1 : T(0);
        dc[2] = T(0.5) * (dcb + dct);
        // cn = sum_m D2_m dc_m (sum_p G[p][m] dc_p)
        T cn = T(0), cd = T(0);
#pragma unroll
        for (int m = 0; m < 3; ++m) cn += D2[m] * dc[m] * (G[0][m] * dc[0] + G[1][m] * dc[1] + G[2][m] * dc[2]);
#pragma unroll
        for (int p = 0; p < 3; ++p) cd += dc[p] * dc[p];
        T kap = (cd > T(0)) ? -a.C_amd * cn / cd : T(0);
        a.kap[t][id] = kap > T(0) ? kap : T(0);
      }
    }
    // advance
    u0 = un0; u1 = un1; v0 = vn0; v1 = vn1;
    w00 = w01; wm0 = wm1; wp0 = wp1; w0m = w0m1; w0p = w0p1;
    dudz_lo0 = dudz_hi0; dudz_lo1 = dudz_hi1; dvdz_lo0 = dvdz_hi0; dvdz_lo1 = dvdz_hi1;
    Uk = U1; Vk = V1; Wk = W1;
  }
}

template <typename T, bool SMAG>
struct ClosureK {
  typedef ClosureArgs<T> Payload;
  static constexpr int kThreads = 256, kMinBlocks = sizeof(T) == 4 ? 4 : 2;
  static __device__ __forceinline__ void run(const Payload& a, uint3 bid, uint3 gdim) {
    closure_body<T, SMAG>(a, bid, gdim);
  }
};

template <typename T, bool SMAG>
__global__ void __launch_bounds__(ClosureK<T, SMAG>::kThreads, ClosureK<T, SMAG>::kMinBlocks) k_closure(const ClosureArgs<T> a) {
  closure_body<T, SMAG>(a, blockIdx, gridDim);
}

template <typename T>
cudaError_t launch_closure(const ClosureArgs<T>& a, cudaStream_t s) {
  // 256-thread blocks of 32 x 8 columns; narrower for grids under 32 columns wide
  int bx = 32;
  while (bx > 1 && bx / 2 >= a.Nx) bx /= 2;
  dim3 blk(bx, 256 / bx);
  // z chunks so that small horizontal grids still fill the GPU (about a million threads), each
  // chunk at least 16 levels deep
  const long long cols = (long long)a.Nx * a.Ny;
  int nch = (int)((1000000 + cols - 1) / cols);
  nch = std::max(1, std::min(nch, a.Nz / 16));
  dim3 grid((a.Nx + blk.x - 1) / blk.x, (a.Ny + blk.y - 1) / blk.y, nch);
  if (a.closure == OCN_CLOSURE_SMAGORINSKY) {
    if (record_launch<ClosureK<T, true>>(a, grid, blk, 0, OCN_K_CLOSURE)) return cudaSuccess;
    k_closure<T, true><<<grid, blk, 0, s>>>(a);
  } else {
    if (record_launch<ClosureK<T, false>>(a, grid, blk, 0, OCN_K_CLOSURE)) return cudaSuccess;
    k_closure<T, false><<<grid, blk, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template cudaError_t launch_closure<float>(const ClosureArgs<float>&, cudaStream_t);
template cudaError_t launch_closure<double>(const ClosureArgs<double>&, cudaStream_t);

}  // namespace ocn
