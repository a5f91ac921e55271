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

// ---------------------------------------------------------------- completion counter
// "Last block" detection: every block publishes its partial result with a
// plain store, then increments a device-scope counter with acquire-release
// semantics (no sequentially consistent fence); the block that sees
// count == gridDim - 1 has acquired every other block's partial.
__device__ __forceinline__ unsigned int atomic_add_acq_rel(unsigned int *p, unsigned int v) {
    unsigned int old;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
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

// ---------------------------------------------------------------- double-float dot accumulation
// FP64 instructions are scarce on this part (2 DFMA/clk/SM), so dot products
// of FP32 vectors are accumulated in "double-float" form: an unevaluated sum
// hi + lo of two floats, updated with Knuth's error-free TwoSum and the
// FMA-based exact product (Dekker / Ogita-Rump-Oishi "Dot2").  The result is
// as accurate as a sum carried in twice the FP32 precision; it is converted to
// FP64 once per warp and the per-warp values are summed in FP64 in a fixed
// order.  The intrinsics below are never contracted or reassociated.
struct DotF {
    float hi = 0.f, lo = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float s = __fadd_rn(hi, v);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(v, bb));
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    __device__ __forceinline__ void add_prod(float a, float b) {
        const float p = __fmul_rn(a, b);
        const float pe = __fmaf_rn(a, b, -p);
        const float s = __fadd_rn(hi, p);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(e, pe));
    }
    __device__ __forceinline__ void merge(float h2, float l2) {
        const float s = __fadd_rn(hi, h2);
        const float bb = __fsub_rn(s, hi);
        const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
        hi = s;
        lo = __fadd_rn(__fadd_rn(lo, l2), e);
    }
};
// FP64 accumulator with the same interface (FP64 vectors).
struct DotD {
    double v = 0.0;
    __device__ __forceinline__ void add(double x) { v += x; }
    __device__ __forceinline__ void add_prod(double a, double b) { v = fma(a, b, v); }
};
template <typename T> struct DotOf;
template <> struct DotOf<float> { using type = DotF; };
template <> struct DotOf<double> { using type = DotD; };

// Block-wide sum of accumulators in a fixed order; all threads get the FP64
// result.  `red` holds >= 32 doubles.
__device__ __forceinline__ double block_sum(const DotF &a, double *red) {
    float hi = a.hi, lo = a.lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        DotF t;
        t.hi = hi;
        t.lo = lo;
        t.merge(h2, l2);
        hi = t.hi;
        lo = t.lo;
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = (double)hi + (double)lo;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += red[w];
        red[32] = t;
    }
    __syncthreads();
    const double r = red[32];
    __syncthreads();
    return r;
}
__device__ __forceinline__ double block_sum(const DotD &a, double *red) { return block_sum(a.v, red); }

// N block sums (N <= 3) with one set of barriers; each result is bitwise the
// one block_sum gives (same per-warp values, same fixed-order sums).  Blocks
// of at most 256 threads; `red` holds >= 34 doubles.
__device__ __forceinline__ float2 warp_dotf(const DotF &a) {
    float hi = a.hi, lo = a.lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        DotF t;
        t.hi = hi;
        t.lo = lo;
        t.merge(h2, l2);
        hi = t.hi;
        lo = t.lo;
    }
    return make_float2(hi, lo);
}
template <int N>
__device__ __forceinline__ void block_sum_n(const DotF *a, double *red, double *out) {
    float2 w[N];
#pragma unroll
    for (int k = 0; k < N; ++k) w[k] = warp_dotf(a[k]);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) red[8 * k + wid] = (double)w[k].x + (double)w[k].y;
    }
    __syncthreads();
    if (lane == 0 && wid < N) {
        double t = 0.0;
        for (int v = 0; v < nw; ++v) t += red[8 * wid + v];
        red[24 + wid] = t;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) out[k] = red[24 + k];
    __syncthreads();
}
__device__ __forceinline__ void block_sum2(const DotF &a, const DotF &b, double *red, double &ra, double &rb) {
    const DotF v[2] = {a, b};
    double o[2];
    block_sum_n<2>(v, red, o);
    ra = o[0];
    rb = o[1];
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

// One thread evaluates a whole patch (layout.h): element j is (a, b, r_j,
// r_{j+1}) in 3D and (a, r_j, r_{j+1}) in 2D.  With e1 = b - a and
// d_j = r_j - a, the cofactor vectors of element j are
//   c1 = d_j x d_{j+1},  c2 = -(e1 x d_{j+1}),  c3 = e1 x d_j   (3D)
//   c1 = perp(d_{j+1}),  c2 = -perp(d_j), perp(v) = (v.y, -v.x)  (2D)
// so e1 x d_j and the node data of r_j carry over from element j-1 to j.
// Per element: the stiffness and mass formulas above; the diagonal (DIAG)
// takes v = e_i: kc |c_i|^2 and cm (2 S + 4 alpha_i).
// out[slot]: 0 -> a, 1 -> b, 2 + j -> r_j (j = 0..m); other slots untouched.
__device__ __forceinline__ float fdiv_fast(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv_fast(double a, double b) { return a / b; }

// beta*dt^2 of a patch's elements: vector loads, all up front.
template <typename T>
__device__ __forceinline__ void load_bd(const T *__restrict__ bdt2, T (&bd)[kPatchMax]) {
    if (sizeof(T) == 4) {
        const float2 *b2 = reinterpret_cast<const float2 *>(bdt2);
#pragma unroll
        for (int k = 0; k < kPatchMax / 2; ++k) {
            const float2 v = __ldg(b2 + k);
            bd[2 * k] = (T)v.x;
            bd[2 * k + 1] = (T)v.y;
        }
    } else {
        const double2 *b2 = reinterpret_cast<const double2 *>(bdt2);
#pragma unroll
        for (int k = 0; k < kPatchMax / 2; ++k) {
            const double2 v = __ldg(b2 + k);
            bd[2 * k] = (T)v.x;
            bd[2 * k + 1] = (T)v.y;
        }
    }
}

// lumped: the mass term by vertex quadrature (int alpha_h phi_i phi_j ~
// delta_ij alpha_i |T| / (d+1) per element: the mass-lumped variant), else
// the consistent form above.
template <int D, typename T, typename N4, bool DIAG, bool LUMP = false>
__device__ __forceinline__ void patch_eval(const N4 *__restrict__ s_node, const T *__restrict__ s_val,
                                           const uint16_t *__restrict__ rec, const T (&bd)[kPatchMax],
                                           T *__restrict__ out) {
    constexpr bool lumped = LUMP;
    // the 24-byte record as three 8-byte loads: [m, a, b, r0], [r1..r4], [r5, r6, -, -]
    const ushort4 q0 = reinterpret_cast<const ushort4 *>(rec)[0];
    const ushort4 q1 = reinterpret_cast<const ushort4 *>(rec)[1];
    const ushort4 q2 = reinterpret_cast<const ushort4 *>(rec)[2];
    const int pm = q0.x;
    const int ring[7] = {q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y};
    const int ia = q0.y;
    const N4 A = s_node[ia];
    const T va = DIAG ? T(0) : s_val[ia];
    const T aa = fabs(A.w);
    T acc_a = T(0), acc_b = T(0);
    if (D == 3) {
        const int ib = q0.z;
        const N4 B = s_node[ib];
        const T vb = DIAG ? T(0) : s_val[ib];
        const T ab = fabs(B.w);
        const T e1x = B.x - A.x, e1y = B.y - A.y, e1z = B.z - A.z;
        N4 R0 = s_node[ring[0]];
        T v0 = DIAG ? T(0) : s_val[ring[0]];
        T d0x = R0.x - A.x, d0y = R0.y - A.y, d0z = R0.z - A.z;
        T w0x = e1y * d0z - e1z * d0y, w0y = e1z * d0x - e1x * d0z, w0z = e1x * d0y - e1y * d0x;
        T acc_c = T(0);
#pragma unroll
        for (int j = 0; j < kPatchMax; ++j) {
            if (j >= pm) break;
            const N4 R1 = s_node[ring[j + 1]];
            const T v1 = DIAG ? T(0) : s_val[ring[j + 1]];
            const T d1x = R1.x - A.x, d1y = R1.y - A.y, d1z = R1.z - A.z;
            const T w1x = e1y * d1z - e1z * d1y, w1y = e1z * d1x - e1x * d1z, w1z = e1x * d1y - e1y * d1x;
            const T c1x = d0y * d1z - d0z * d1y, c1y = d0z * d1x - d0x * d1z, c1z = d0x * d1y - d0y * d1x;
            const T ad = fabs(e1x * c1x + e1y * c1y + e1z * c1z);
            const T kc = fdiv_fast(bd[j], T(6) * ad);
            const T a2 = fabs(R0.w), a3 = fabs(R1.w);
            const T S = (aa + ab) + (a2 + a3);
            const T cm = ad * T(1.0 / 720.0);
            T o0, o1, o2, o3;
            if (DIAG) {
                const T c0x = -(c1x - w1x + w0x), c0y = -(c1y - w1y + w0y), c0z = -(c1z - w1z + w0z);
                const T cl = ad * T(1.0 / 24.0);
                o0 = (lumped ? cl * aa : cm * (T(2) * S + T(4) * aa)) + kc * (c0x * c0x + c0y * c0y + c0z * c0z);
                o1 = (lumped ? cl * ab : cm * (T(2) * S + T(4) * ab)) + kc * (c1x * c1x + c1y * c1y + c1z * c1z);
                o2 = (lumped ? cl * a2 : cm * (T(2) * S + T(4) * a2)) + kc * (w1x * w1x + w1y * w1y + w1z * w1z);
                o3 = (lumped ? cl * a3 : cm * (T(2) * S + T(4) * a3)) + kc * (w0x * w0x + w0y * w0y + w0z * w0z);
            } else {
                // g = (vb - va) c1 + (v0 - va) c2 + (v1 - va) c3, c2 = -w1, c3 = w0
                const T t1 = vb - va, t2 = v0 - va, t3 = v1 - va;
                const T gx = t1 * c1x - t2 * w1x + t3 * w0x;
                const T gy = t1 * c1y - t2 * w1y + t3 * w0y;
                const T gz = t1 * c1z - t2 * w1z + t3 * w0z;
                const T k1 = kc * (c1x * gx + c1y * gy + c1z * gz);
                const T k2 = -kc * (w1x * gx + w1y * gy + w1z * gz);
                const T k3 = kc * (w0x * gx + w0y * gy + w0z * gz);
                const T k0 = -(k1 + k2 + k3);
                if constexpr (lumped) {
                    const T cl = ad * T(1.0 / 24.0);
                    o0 = cl * aa * va + k0;
                    o1 = cl * ab * vb + k1;
                    o2 = cl * a2 * v0 + k2;
                    o3 = cl * a3 * v1 + k3;
                } else {
                    const T X = (va + vb) + (v0 + v1);
                    const T Q = (aa * va + ab * vb) + (a2 * v0 + a3 * v1);
                    const T base = S * X + Q;
                    o0 = cm * (base + S * va + aa * (X + T(2) * va)) + k0;
                    o1 = cm * (base + S * vb + ab * (X + T(2) * vb)) + k1;
                    o2 = cm * (base + S * v0 + a2 * (X + T(2) * v0)) + k2;
                    o3 = cm * (base + S * v1 + a3 * (X + T(2) * v1)) + k3;
                }
            }
            acc_a += o0;
            acc_b += o1;
            out[2 + j] = acc_c + o2;
            acc_c = o3;
            d0x = d1x; d0y = d1y; d0z = d1z;
            w0x = w1x; w0y = w1y; w0z = w1z;
            R0 = R1;
            v0 = v1;
        }
        out[2 + pm] = acc_c;
        out[0] = acc_a;
        out[1] = acc_b;
    } else {
        N4 R0 = s_node[ring[0]];
        T v0 = DIAG ? T(0) : s_val[ring[0]];
        T d0x = R0.x - A.x, d0y = R0.y - A.y;
        T acc_c = T(0);
#pragma unroll
        for (int j = 0; j < kPatchMax; ++j) {
            if (j >= pm) break;
            const N4 R1 = s_node[ring[j + 1]];
            const T v1 = DIAG ? T(0) : s_val[ring[j + 1]];
            const T d1x = R1.x - A.x, d1y = R1.y - A.y;
            // c1 = perp(d1) = (d1y, -d1x), c2 = -perp(d0) = (-d0y, d0x)
            const T c1x = d1y, c1y = -d1x, c2x = -d0y, c2y = d0x;
            const T ad = fabs(d0x * d1y - d0y * d1x);
            const T kc = fdiv_fast(bd[j], T(2) * ad);
            const T a1 = fabs(R0.w), a2 = fabs(R1.w);
            const T S = aa + a1 + a2;
            const T cm = ad * T(1.0 / 120.0);
            T o0, o1, o2;
            if (DIAG) {
                const T c0x = -(c1x + c2x), c0y = -(c1y + c2y);
                const T cl = ad * T(1.0 / 6.0);
                o0 = (lumped ? cl * aa : cm * (T(2) * S + T(4) * aa)) + kc * (c0x * c0x + c0y * c0y);
                o1 = (lumped ? cl * a1 : cm * (T(2) * S + T(4) * a1)) + kc * (c1x * c1x + c1y * c1y);
                o2 = (lumped ? cl * a2 : cm * (T(2) * S + T(4) * a2)) + kc * (c2x * c2x + c2y * c2y);
            } else {
                const T t1 = v0 - va, t2 = v1 - va;
                const T gx = t1 * c1x + t2 * c2x, gy = t1 * c1y + t2 * c2y;
                const T k1 = kc * (c1x * gx + c1y * gy);
                const T k2 = kc * (c2x * gx + c2y * gy);
                const T k0 = -(k1 + k2);
                if constexpr (lumped) {
                    const T cl = ad * T(1.0 / 6.0);
                    o0 = cl * aa * va + k0;
                    o1 = cl * a1 * v0 + k1;
                    o2 = cl * a2 * v1 + k2;
                } else {
                    const T X = va + v0 + v1, Q = aa * va + a1 * v0 + a2 * v1;
                    const T base = S * X + Q;
                    o0 = cm * (base + S * va + aa * (X + T(2) * va)) + k0;
                    o1 = cm * (base + S * v0 + a1 * (X + T(2) * v0)) + k1;
                    o2 = cm * (base + S * v1 + a2 * (X + T(2) * v1)) + k2;
                }
            }
            acc_a += o0;
            out[2 + j] = acc_c + o1;
            acc_c = o2;
            d0x = d1x; d0y = d1y;
            R0 = R1;
            v0 = v1;
        }
        out[2 + pm] = acc_c;
        out[0] = acc_a;
    }
}

// FP64 evaluation of one star patch from geometry computed once per mesh on
// the host (mesh upload): for every element slot the symmetric stiffness
// weights G_ab = c_a.c_b / (d! |det|) of its vertex pairs (K^e_ab = beta G_ab)
// and |det|.  The element arithmetic per tet drops to differences, products
// and sums (no cross products, no division), which is what matters on a GPU
// whose FP64 rate is a small fraction of its FP32 rate.  The result equals
// patch_eval<D, double, ...> up to rounding.
// Slot layout, 3D (8 doubles): G_AB, G_A0, G_A1, G_B0, G_B1, G_01, |det|, 0
// with A, B the patch's edge and 0, 1 ring nodes j, j+1; 2D (4 doubles):
// G_A0, G_A1, G_01, |det|.  Rows of G sum to zero (sum_a c_a = 0), so
// (K^e v)_a = beta sum_b G_ab (v_b - v_a) and G_aa = -sum_{b != a} G_ab.
template <int D, bool DIAG, bool LUMP>
__device__ __forceinline__ void patch_eval_geo(const NodeD *__restrict__ s_node, const double *__restrict__ s_val,
                                               const uint16_t *__restrict__ rec, const double (&bd)[kPatchMax],
                                               const double *__restrict__ geo, double *__restrict__ out) {
    const ushort4 q0 = reinterpret_cast<const ushort4 *>(rec)[0];
    const ushort4 q1 = reinterpret_cast<const ushort4 *>(rec)[1];
    const ushort4 q2 = reinterpret_cast<const ushort4 *>(rec)[2];
    const int pm = q0.x;
    const int ring[7] = {q0.w, q1.x, q1.y, q1.z, q1.w, q2.x, q2.y};
    const int ia = q0.y;
    const double aa = fabs(s_node[ia].w);
    const double va = DIAG ? 0.0 : s_val[ia];
    double acc_a = 0.0, acc_b = 0.0, acc_c = 0.0;
    if (D == 3) {
        const int ib = q0.z;
        const double ab = fabs(s_node[ib].w);
        const double vb = DIAG ? 0.0 : s_val[ib];
        double a2 = fabs(s_node[ring[0]].w);
        double v0 = DIAG ? 0.0 : s_val[ring[0]];
        const double2 *g2 = reinterpret_cast<const double2 *>(geo);
#pragma unroll
        for (int j = 0; j < kPatchMax; ++j) {
            if (j >= pm) break;
            const double2 g0 = __ldg(g2 + 4 * j), g1 = __ldg(g2 + 4 * j + 1), gg = __ldg(g2 + 4 * j + 2),
                          g3 = __ldg(g2 + 4 * j + 3);
            const double gAB = g0.x, gA0 = g0.y, gA1 = g1.x, gB0 = g1.y, gB1 = gg.x, g01 = gg.y, ad = g3.x;
            const int r1 = ring[j + 1];
            const double a3 = fabs(s_node[r1].w);
            const double v1 = DIAG ? 0.0 : s_val[r1];
            const double b = bd[j];
            double o0, o1, o2, o3;
            if (DIAG) {
                const double kA = -(gAB + gA0 + gA1), kB = -(gAB + gB0 + gB1), k0 = -(gA0 + gB0 + g01),
                             k1 = -(gA1 + gB1 + g01);
                if (LUMP) {
                    const double cl = ad * (1.0 / 24.0);
                    o0 = cl * aa + b * kA;
                    o1 = cl * ab + b * kB;
                    o2 = cl * a2 + b * k0;
                    o3 = cl * a3 + b * k1;
                } else {
                    const double cm = ad * (1.0 / 720.0);
                    const double S = (aa + ab) + (a2 + a3);
                    o0 = cm * (2.0 * S + 4.0 * aa) + b * kA;
                    o1 = cm * (2.0 * S + 4.0 * ab) + b * kB;
                    o2 = cm * (2.0 * S + 4.0 * a2) + b * k0;
                    o3 = cm * (2.0 * S + 4.0 * a3) + b * k1;
                }
            } else {
                const double wAB = gAB * (vb - va), wA0 = gA0 * (v0 - va), wA1 = gA1 * (v1 - va);
                const double wB0 = gB0 * (v0 - vb), wB1 = gB1 * (v1 - vb), w01 = g01 * (v1 - v0);
                const double kA = b * ((wAB + wA0) + wA1);
                const double kB = b * ((wB0 + wB1) - wAB);
                const double k0 = b * (w01 - (wA0 + wB0));
                const double k1 = -b * ((wA1 + wB1) + w01);
                if (LUMP) {
                    const double cl = ad * (1.0 / 24.0);
                    o0 = cl * aa * va + kA;
                    o1 = cl * ab * vb + kB;
                    o2 = cl * a2 * v0 + k0;
                    o3 = cl * a3 * v1 + k1;
                } else {
                    const double cm = ad * (1.0 / 720.0);
                    const double S = (aa + ab) + (a2 + a3);
                    const double X = (va + vb) + (v0 + v1);
                    const double Q = (aa * va + ab * vb) + (a2 * v0 + a3 * v1);
                    const double base = S * X + Q;
                    o0 = cm * (base + S * va + aa * (X + 2.0 * va)) + kA;
                    o1 = cm * (base + S * vb + ab * (X + 2.0 * vb)) + kB;
                    o2 = cm * (base + S * v0 + a2 * (X + 2.0 * v0)) + k0;
                    o3 = cm * (base + S * v1 + a3 * (X + 2.0 * v1)) + k1;
                }
            }
            acc_a += o0;
            acc_b += o1;
            out[2 + j] = acc_c + o2;
            acc_c = o3;
            a2 = a3;
            v0 = v1;
        }
        out[2 + pm] = acc_c;
        out[0] = acc_a;
        out[1] = acc_b;
    } else {
        double a1 = fabs(s_node[ring[0]].w);
        double v0 = DIAG ? 0.0 : s_val[ring[0]];
        const double2 *g2 = reinterpret_cast<const double2 *>(geo);
#pragma unroll
        for (int j = 0; j < kPatchMax; ++j) {
            if (j >= pm) break;
            const double2 g0 = __ldg(g2 + 2 * j), g1 = __ldg(g2 + 2 * j + 1);
            const double gA0 = g0.x, gA1 = g0.y, g01 = g1.x, ad = g1.y;
            const int r1 = ring[j + 1];
            const double a2 = fabs(s_node[r1].w);
            const double v1 = DIAG ? 0.0 : s_val[r1];
            const double b = bd[j];
            double o0, o1, o2;
            if (DIAG) {
                const double kA = -(gA0 + gA1), k0 = -(gA0 + g01), k1 = -(gA1 + g01);
                if (LUMP) {
                    const double cl = ad * (1.0 / 6.0);
                    o0 = cl * aa + b * kA;
                    o1 = cl * a1 + b * k0;
                    o2 = cl * a2 + b * k1;
                } else {
                    const double cm = ad * (1.0 / 120.0);
                    const double S = aa + a1 + a2;
                    o0 = cm * (2.0 * S + 4.0 * aa) + b * kA;
                    o1 = cm * (2.0 * S + 4.0 * a1) + b * k0;
                    o2 = cm * (2.0 * S + 4.0 * a2) + b * k1;
                }
            } else {
                const double wA0 = gA0 * (v0 - va), wA1 = gA1 * (v1 - va), w01 = g01 * (v1 - v0);
                const double kA = b * (wA0 + wA1);
                const double k0 = b * (w01 - wA0);
                const double k1 = -b * (wA1 + w01);
                if (LUMP) {
                    const double cl = ad * (1.0 / 6.0);
                    o0 = cl * aa * va + kA;
                    o1 = cl * a1 * v0 + k0;
                    o2 = cl * a2 * v1 + k1;
                } else {
                    const double cm = ad * (1.0 / 120.0);
                    const double S = aa + a1 + a2;
                    const double X = va + v0 + v1, Q = aa * va + a1 * v0 + a2 * v1;
                    const double base = S * X + Q;
                    o0 = cm * (base + S * va + aa * (X + 2.0 * va)) + kA;
                    o1 = cm * (base + S * v0 + a1 * (X + 2.0 * v0)) + k0;
                    o2 = cm * (base + S * v1 + a2 * (X + 2.0 * v1)) + k1;
                }
            }
            acc_a += o0;
            out[2 + j] = acc_c + o1;
            acc_c = o2;
            a1 = a2;
            v0 = v1;
        }
        out[2 + pm] = acc_c;
        out[0] = acc_a;
    }
}

}  // namespace ps
