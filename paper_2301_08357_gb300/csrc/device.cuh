// Device-side building blocks for sm_103a: PTX wrappers for mbarriers and
// bulk (TMA engine) copies, the P1 element kernels, and block reductions.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "layout.h"

namespace ps {

// Bounded waits: an mbarrier wait gives up after this many try_wait rounds
// (each round may itself suspend for a hardware-defined time slice) and a grid
// barrier after this many polls; both then record an error and return.
constexpr uint32_t kMbarSpinLimit = 1u << 22;
constexpr uint32_t kGridSpinLimit = 1u << 26;

enum DevErr : int { kErrNone = 0, kErrMbarTimeout = 1, kErrGridTimeout = 2, kErrBadSize = 4 };

// Node record staged per chunk: coordinates relative to the chunk origin in
// x, y, z (z = 0 in 2D) and alpha in w, with the sign bit of w set on
// Dirichlet nodes (alpha itself is >= 0).
struct alignas(16) NodeF { float x, y, z, w; };
struct alignas(32) NodeD { double x, y, z, w; };
template <typename T> struct NodeOf;
template <> struct NodeOf<float> { using type = NodeF; };
template <> struct NodeOf<double> { using type = NodeD; };

__device__ __forceinline__ bool is_dirichlet(float w) { return __float_as_int(w) < 0; }
__device__ __forceinline__ bool is_dirichlet(double w) { return __double_as_longlong(w) < 0; }

// ---------------------------------------------------------------- PTX: mbarrier + bulk copy
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Global -> shared bulk copy through the TMA engine; completion is signalled
// on `bar` as transaction bytes.  dst, src 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of `bar`.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    for (uint32_t i = 0; i < kMbarSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// ---------------------------------------------------------------- reductions
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
// Block-wide sum in a fixed order (the result is bitwise reproducible for a
// given blockDim).  `red` holds >= 32 doubles.  All threads get the result.
__device__ __forceinline__ double block_sum(double v, double *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
    if (wid == 0) t = warp_sum(t);
    if (threadIdx.x == 0) red[0] = t;
    __syncthreads();
    double r = red[0];
    __syncthreads();
    return r;
}
// Sum of n doubles in global memory in a fixed order, by one block.
__device__ __forceinline__ double block_sum_array(const double *a, int n, double *red) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += __ldcg(a + i);
    return block_sum(s, red);
}

// ---------------------------------------------------------------- P1 element kernels
// Notation: vertices p0..pd with coordinates (x,y[,z]) and nodal alpha in w;
// nodal values v0..vd; bdt2 = beta_e * dt^2.  Jacobian columns e_k = p_k - p0,
// cofactor vectors c_k with grad(lambda_k) = c_k / det (k = 1..d) and
// c_0 = -(c_1 + ... + c_d); |T| = |det| / d!.
//   stiffness:  (K v)_i = beta |T| grad(lambda_i) . grad(v_h)
//                       = bdt2 / (d! |det|) * c_i . g,   g = sum_k (v_k - v_0) c_k
//   mass:       (M_alpha v)_i = sum_jk alpha_k v_j int lambda_i lambda_j lambda_k
//                 = cm (S X + Q + S v_i + alpha_i (X + 2 v_i)),
//               S = sum alpha_k, X = sum v_k, Q = sum alpha_k v_k,
//               cm = |T| d! / (d+3)!  (= |det|/720 in 3D, |det|/120 in 2D),
//   from int lambda^a = d! |T| prod(a_i!) / (d + sum a_i)!.

template <typename T, typename N4>
__device__ __forceinline__ void elem_apply_3d(const N4 &p0, const N4 &p1, const N4 &p2, const N4 &p3, T v0,
                                              T v1, T v2, T v3, T bdt2, T &o0, T &o1, T &o2, T &o3) {
    const T e1x = p1.x - p0.x, e1y = p1.y - p0.y, e1z = p1.z - p0.z;
    const T e2x = p2.x - p0.x, e2y = p2.y - p0.y, e2z = p2.z - p0.z;
    const T e3x = p3.x - p0.x, e3y = p3.y - p0.y, e3z = p3.z - p0.z;
    const T c1x = e2y * e3z - e2z * e3y, c1y = e2z * e3x - e2x * e3z, c1z = e2x * e3y - e2y * e3x;
    const T c2x = e3y * e1z - e3z * e1y, c2y = e3z * e1x - e3x * e1z, c2z = e3x * e1y - e3y * e1x;
    const T c3x = e1y * e2z - e1z * e2y, c3y = e1z * e2x - e1x * e2z, c3z = e1x * e2y - e1y * e2x;
    const T ad = fabs(e1x * c1x + e1y * c1y + e1z * c1z);
    const T d1 = v1 - v0, d2 = v2 - v0, d3 = v3 - v0;
    const T gx = d1 * c1x + d2 * c2x + d3 * c3x;
    const T gy = d1 * c1y + d2 * c2y + d3 * c3y;
    const T gz = d1 * c1z + d2 * c2z + d3 * c3z;
    const T kc = bdt2 / (T(6) * ad);
    const T k1 = kc * (c1x * gx + c1y * gy + c1z * gz);
    const T k2 = kc * (c2x * gx + c2y * gy + c2z * gz);
    const T k3 = kc * (c3x * gx + c3y * gy + c3z * gz);
    const T k0 = -(k1 + k2 + k3);
    const T a0 = fabs(p0.w), a1 = fabs(p1.w), a2 = fabs(p2.w), a3 = fabs(p3.w);
    const T S = (a0 + a1) + (a2 + a3);
    const T X = (v0 + v1) + (v2 + v3);
    const T Q = (a0 * v0 + a1 * v1) + (a2 * v2 + a3 * v3);
    const T cm = ad * T(1.0 / 720.0);
    const T base = S * X + Q;
    o0 = cm * (base + S * v0 + a0 * (X + T(2) * v0)) + k0;
    o1 = cm * (base + S * v1 + a1 * (X + T(2) * v1)) + k1;
    o2 = cm * (base + S * v2 + a2 * (X + T(2) * v2)) + k2;
    o3 = cm * (base + S * v3 + a3 * (X + T(2) * v3)) + k3;
}

template <typename T, typename N4>
__device__ __forceinline__ void elem_apply_2d(const N4 &p0, const N4 &p1, const N4 &p2, T v0, T v1, T v2,
                                              T bdt2, T &o0, T &o1, T &o2) {
    const T e1x = p1.x - p0.x, e1y = p1.y - p0.y;
    const T e2x = p2.x - p0.x, e2y = p2.y - p0.y;
    const T c1x = e2y, c1y = -e2x, c2x = -e1y, c2y = e1x;
    const T ad = fabs(e1x * e2y - e1y * e2x);
    const T d1 = v1 - v0, d2 = v2 - v0;
    const T gx = d1 * c1x + d2 * c2x, gy = d1 * c1y + d2 * c2y;
    const T kc = bdt2 / (T(2) * ad);
    const T k1 = kc * (c1x * gx + c1y * gy);
    const T k2 = kc * (c2x * gx + c2y * gy);
    const T k0 = -(k1 + k2);
    const T a0 = fabs(p0.w), a1 = fabs(p1.w), a2 = fabs(p2.w);
    const T S = a0 + a1 + a2, X = v0 + v1 + v2, Q = a0 * v0 + a1 * v1 + a2 * v2;
    const T cm = ad * T(1.0 / 120.0);
    const T base = S * X + Q;
    o0 = cm * (base + S * v0 + a0 * (X + T(2) * v0)) + k0;
    o1 = cm * (base + S * v1 + a1 * (X + T(2) * v1)) + k1;
    o2 = cm * (base + S * v2 + a2 * (X + T(2) * v2)) + k2;
}

// Diagonal entries of the element matrix: cm (2 S + 4 alpha_i) + bdt2 |c_i|^2 / (d! |det|).
template <typename T, typename N4>
__device__ __forceinline__ void elem_diag_3d(const N4 &p0, const N4 &p1, const N4 &p2, const N4 &p3, T bdt2,
                                             T &o0, T &o1, T &o2, T &o3) {
    const T e1x = p1.x - p0.x, e1y = p1.y - p0.y, e1z = p1.z - p0.z;
    const T e2x = p2.x - p0.x, e2y = p2.y - p0.y, e2z = p2.z - p0.z;
    const T e3x = p3.x - p0.x, e3y = p3.y - p0.y, e3z = p3.z - p0.z;
    const T c1x = e2y * e3z - e2z * e3y, c1y = e2z * e3x - e2x * e3z, c1z = e2x * e3y - e2y * e3x;
    const T c2x = e3y * e1z - e3z * e1y, c2y = e3z * e1x - e3x * e1z, c2z = e3x * e1y - e3y * e1x;
    const T c3x = e1y * e2z - e1z * e2y, c3y = e1z * e2x - e1x * e2z, c3z = e1x * e2y - e1y * e2x;
    const T c0x = -(c1x + c2x + c3x), c0y = -(c1y + c2y + c3y), c0z = -(c1z + c2z + c3z);
    const T ad = fabs(e1x * c1x + e1y * c1y + e1z * c1z);
    const T kc = bdt2 / (T(6) * ad);
    const T a0 = fabs(p0.w), a1 = fabs(p1.w), a2 = fabs(p2.w), a3 = fabs(p3.w);
    const T S = (a0 + a1) + (a2 + a3);
    const T cm = ad * T(1.0 / 720.0);
    o0 = cm * (T(2) * S + T(4) * a0) + kc * (c0x * c0x + c0y * c0y + c0z * c0z);
    o1 = cm * (T(2) * S + T(4) * a1) + kc * (c1x * c1x + c1y * c1y + c1z * c1z);
    o2 = cm * (T(2) * S + T(4) * a2) + kc * (c2x * c2x + c2y * c2y + c2z * c2z);
    o3 = cm * (T(2) * S + T(4) * a3) + kc * (c3x * c3x + c3y * c3y + c3z * c3z);
}

template <typename T, typename N4>
__device__ __forceinline__ void elem_diag_2d(const N4 &p0, const N4 &p1, const N4 &p2, T bdt2, T &o0, T &o1,
                                             T &o2) {
    const T e1x = p1.x - p0.x, e1y = p1.y - p0.y;
    const T e2x = p2.x - p0.x, e2y = p2.y - p0.y;
    const T c1x = e2y, c1y = -e2x, c2x = -e1y, c2y = e1x;
    const T c0x = -(c1x + c2x), c0y = -(c1y + c2y);
    const T ad = fabs(e1x * e2y - e1y * e2x);
    const T kc = bdt2 / (T(2) * ad);
    const T a0 = fabs(p0.w), a1 = fabs(p1.w), a2 = fabs(p2.w);
    const T S = a0 + a1 + a2;
    const T cm = ad * T(1.0 / 120.0);
    o0 = cm * (T(2) * S + T(4) * a0) + kc * (c0x * c0x + c0y * c0y);
    o1 = cm * (T(2) * S + T(4) * a1) + kc * (c1x * c1x + c1y * c1y);
    o2 = cm * (T(2) * S + T(4) * a2) + kc * (c2x * c2x + c2y * c2y);
}

}  // namespace ps
