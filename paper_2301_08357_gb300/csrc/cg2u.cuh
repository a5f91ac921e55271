// FP32 CG operator kernel of 3D meshes on paired patches (layout.h, "units").
//
// The same iteration step as k_cg2_chunks<3, float> (p = D^-1 r + beta p on
// the chunk's nodes, q = A p, the chunk's share of p.Ap), organised for the
// instruction budget of a pass that moves ~20 bytes per tetrahedron:
//   * one thread evaluates one unit -- two star patches of equal size -- with
//     packed FP32x2 arithmetic (FFMA2 / FADD2 / FMUL2: one instruction for both
//     patches), so each element costs about half the issue slots;
//   * the chunk's node records, unit records, beta*dt^2/6 values and
//     shared-node destinations are staged into shared memory by bulk copies
//     (one mbarrier); a thread reads its unit's record words and
//     coefficients from there as its elements need them, so they hold no
//     registers across the unit;
//   * coordinates enter the arithmetic as differences to the unit's node a
//     (scalar subtractions into the packed operands), and a duplicate second
//     half is dropped by a zero scale, not a branch;
//   * contributions are added into per-node fixed-point sums in shared
//     memory (32-bit integer atomics: exact, so the result does not depend on
//     the order of the additions -- no incidence list, bitwise reproducible);
//     the chunk's scale comes from a bound on every partial sum (below), and
//     each node sum is rounded to FP32 once;
//   * shared nodes' inputs come from a chunk-major halo, contiguous per chunk;
//     a thread has all its nodes' loads in flight before any store;
//   * the chunk's p.Ap share is merged per warp and then across the four
//     warps by one thread; the chunk block stores it and exits, and one
//     extra block of the grid sums the shares in chunk order and sets alpha
//     (no fence, counter or wait in the chunk blocks).
// Scale of the fixed-point sums: element matrices are positive semidefinite
// (mass with alpha >= 0, stiffness with beta > 0), so |A^e_ij| <=
// sqrt(A^e_ii A^e_jj) <= Dmax, the largest diagonal entry D_jj over the
// chunk's free nodes (Dirichlet columns carry v = 0); a node in at most
// n_star of the chunk's elements therefore has every partial sum bounded by
// B = 4 n_star Dmax vmax, vmax = max |v| over the chunk.  Contributions are
// scaled by 2^(47 - ceil(log2 B)), so every partial sum stays below 2^47 (a
// factor of two below the 2^48 the split into two 32-bit sums allows); the
// resolution, 2^-47 B ~ 7e-15 B, is far below the FP32 rounding of a row for
// any dynamic range below ~1e8 between the chunk's largest and a row's own
// scale.  Each node sum is rounded to FP32 at the end (2^24 h + l in one
// FMA).  Interior Dirichlet rows are masked to 0 whatever their sums (shared
// ones by the update kernel, which sums the partials).  The element
// arithmetic is that of patch_eval (device.cuh): with e1 = b - a and
// d_j = r_j - a, element j of a patch has the cofactor vectors
// c1 = d_j x d_{j+1}, c2 = -(e1 x d_{j+1}), c3 = e1 x d_j and c0 = -(c1+c2+c3),
// det = e1 . c1; stiffness K v = beta dt^2 / (6 |det|) (c_i . g),
// g = sum_k (v_k - v_a) c_k; consistent mass (M_alpha v)_i =
// |det|/720 (S X + Q + S v_i + alpha_i (X + 2 v_i)), S = sum alpha, X = sum v,
// Q = sum alpha v; lumped mass |det|/24 alpha_i v_i.
#pragma once
#include "cg2.cuh"

namespace ps {

// ---------------------------------------------------------------- packed FP32x2
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __fadd2_rn(a, p_neg(b)); }
__device__ __forceinline__ float2 p_abs(float2 a) { return make_float2(fabsf(a.x), fabsf(a.y)); }
__device__ __forceinline__ float2 p_set(float v) { return make_float2(v, v); }
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

struct P3 {
    float2 x, y, z;
};
// a x b
__device__ __forceinline__ P3 p3_cross(const P3 &a, const P3 &b) {
    return {p_fma(a.y, b.z, p_neg(p_mul(a.z, b.y))), p_fma(a.z, b.x, p_neg(p_mul(a.x, b.z))),
            p_fma(a.x, b.y, p_neg(p_mul(a.y, b.x)))};
}
__device__ __forceinline__ float2 p3_dot(const P3 &a, const P3 &b) {
    return p_fma(a.z, b.z, p_fma(a.y, b.y, p_mul(a.x, b.x)));
}

// Node of both halves relative to the unit's node a of each half: the
// coordinate differences p - a (one scalar subtraction per half, written
// straight into the packed operand), alpha (absolute value: the sign bit
// marks Dirichlet nodes) and the input value.
struct PRel {
    P3 d;
    float2 al, v;
};
__device__ __forceinline__ PRel prel(const NodeF *__restrict__ s_node, const float *__restrict__ s_val, uint32_t w,
                                     const float3 &a0, const float3 &a1) {
    const int i0 = (int)(w & 0xffffu), i1 = (int)(w >> 16);
    const NodeF n0 = s_node[i0], n1 = s_node[i1];
    PRel r;
    r.d = {make_float2(n0.x - a0.x, n1.x - a1.x), make_float2(n0.y - a0.y, n1.y - a1.y),
           make_float2(n0.z - a0.z, n1.z - a1.z)};
    r.al = make_float2(fabsf(n0.w), fabsf(n1.w));
    r.v = make_float2(s_val[i0], s_val[i1]);
    return r;
}

// Fixed-point node sums: the scaled contribution t (|t| < 2^48, a multiple of
// the resolution after rounding) is split exactly into t = 2^24 h + l with
// integers h = rint(t / 2^24) and |l| <= 2^23; h and l are added to the
// node's two 32-bit integer sums (a node takes at most a few dozen
// contributions, so neither overflows).  Only 32-bit conversions and integer
// atomics: all fast paths.
__device__ __forceinline__ void acc_add1(int *__restrict__ s_acc, int i, float t) {
    const float hf = rintf(t * (1.0f / 16777216.0f));
    const float lf = fmaf(-hf, 16777216.0f, t);   // exact: t and 2^24 hf differ by at most 2^23
    atomicAdd(s_acc + 2 * i, __float2int_rn(hf));
    atomicAdd(s_acc + 2 * i + 1, __float2int_rn(lf));
}
// Add a contribution of each half to its node's sums.  S is the chunk's
// scale for both halves, with S.y = 0 on a unit whose second half duplicates
// the first: that half then adds exact zeros (no branch).
__device__ __forceinline__ void acc_add(int *__restrict__ s_acc, uint32_t w, float2 v, float2 S) {
    const float2 t = p_mul(v, S);
    acc_add1(s_acc, (int)(w & 0xffffu), t.x);
    acc_add1(s_acc, (int)(w >> 16), t.y);
}

// One unit of M tetrahedra per half: contributions of node slots a, b and
// r_j (j = 0..M) into the fixed-point sums.  rec: the unit record and bd:
// beta*dt^2/6 of element j of each half, both in shared memory (read as the
// elements need them); S: the scale of each half.
template <int M, bool LUMP>
__device__ __forceinline__ void unit_eval(const NodeF *__restrict__ s_node, const float *__restrict__ s_val,
                                          const uint32_t *__restrict__ rec, const float2 *__restrict__ bd,
                                          int *__restrict__ s_acc, float2 S) {
    const uint32_t wa = rec[1];
    const NodeF na0 = s_node[wa & 0xffffu], na1 = s_node[wa >> 16];
    const float3 a0 = make_float3(na0.x, na0.y, na0.z), a1 = make_float3(na1.x, na1.y, na1.z);
    const float2 Aal = make_float2(fabsf(na0.w), fabsf(na1.w));
    const float2 Av = make_float2(s_val[wa & 0xffffu], s_val[wa >> 16]);
    const PRel B = prel(s_node, s_val, rec[2], a0, a1);
    const P3 e1 = B.d;
    PRel R0 = prel(s_node, s_val, rec[3], a0, a1);
    P3 d0 = R0.d;
    P3 w0 = p3_cross(e1, d0);
    const float2 t1 = p_sub(B.v, Av);
    float2 t2 = p_sub(R0.v, Av);
    const float2 sAB = p_add(Aal, B.al);
    const float2 xAB = p_add(Av, B.v);
    const float2 qa = p_mul(Aal, Av), qb = p_mul(B.al, B.v);
    const float2 qAB = p_add(qa, qb);
    float2 q0 = p_mul(R0.al, R0.v);
    float2 acc_a = p_set(0.f), acc_b = p_set(0.f), acc_c = p_set(0.f);
    const float2 two = p_set(2.f);
#pragma unroll
    for (int j = 0; j < M; ++j) {
        const PRel R1 = prel(s_node, s_val, rec[4 + j], a0, a1);
        const P3 d1 = R1.d;
        const P3 w1 = p3_cross(e1, d1);
        const P3 c1 = p3_cross(d0, d1);
        const float2 ad = p_abs(p3_dot(e1, c1));
        const float2 kc = p_mul(bd[j], make_float2(rcp_approx(ad.x), rcp_approx(ad.y)));
        const float2 t3 = p_sub(R1.v, Av);
        // g = t1 c1 - t2 w1 + t3 w0, scaled by kc
        const float2 nt2 = p_neg(t2);
        P3 g;
        g.x = p_mul(kc, p_fma(t3, w0.x, p_fma(nt2, w1.x, p_mul(t1, c1.x))));
        g.y = p_mul(kc, p_fma(t3, w0.y, p_fma(nt2, w1.y, p_mul(t1, c1.y))));
        g.z = p_mul(kc, p_fma(t3, w0.z, p_fma(nt2, w1.z, p_mul(t1, c1.z))));
        const float2 k1 = p3_dot(c1, g);
        const float2 k2 = p_neg(p3_dot(w1, g));
        const float2 k3 = p3_dot(w0, g);
        const float2 k0 = p_neg(p_add(p_add(k1, k2), k3));
        const float2 q1 = p_mul(R1.al, R1.v);
        float2 o0, o1, o2, o3;
        if constexpr (LUMP) {
            const float2 cl = p_mul(ad, p_set(1.0f / 24.0f));
            o0 = p_fma(cl, qa, k0);
            o1 = p_fma(cl, qb, k1);
            o2 = p_fma(cl, q0, k2);
            o3 = p_fma(cl, q1, k3);
        } else {
            const float2 Ssum = p_add(sAB, p_add(R0.al, R1.al));
            const float2 X = p_add(xAB, p_add(R0.v, R1.v));
            const float2 Q = p_add(qAB, p_add(q0, q1));
            const float2 base = p_fma(Ssum, X, Q);
            const float2 cm = p_mul(ad, p_set(1.0f / 720.0f));
            // o_i = cm (base + S v_i + alpha_i (X + 2 v_i)) + k_i
            o0 = p_fma(cm, p_fma(Aal, p_fma(two, Av, X), p_fma(Ssum, Av, base)), k0);
            o1 = p_fma(cm, p_fma(B.al, p_fma(two, B.v, X), p_fma(Ssum, B.v, base)), k1);
            o2 = p_fma(cm, p_fma(R0.al, p_fma(two, R0.v, X), p_fma(Ssum, R0.v, base)), k2);
            o3 = p_fma(cm, p_fma(R1.al, p_fma(two, R1.v, X), p_fma(Ssum, R1.v, base)), k3);
        }
        acc_a = p_add(acc_a, o0);
        acc_b = p_add(acc_b, o1);
        acc_add(s_acc, rec[3 + j], p_add(acc_c, o2), S);
        acc_c = o3;
        d0 = d1;
        w0 = w1;
        R0 = R1;
        t2 = t3;
        q0 = q1;
    }
    acc_add(s_acc, rec[3 + M], acc_c, S);
    acc_add(s_acc, wa, acc_a, S);
    acc_add(s_acc, rec[2], acc_b, S);
}

template <bool LUMP>
__device__ __forceinline__ void unit_eval_any(const NodeF *__restrict__ s_node, const float *__restrict__ s_val,
                                              const uint32_t *__restrict__ rec, const float2 *__restrict__ bd,
                                              int *__restrict__ s_acc, float2 S) {
    switch (rec[0] & 0xffu) {
        case 6: unit_eval<6, LUMP>(s_node, s_val, rec, bd, s_acc, S); break;
        case 5: unit_eval<5, LUMP>(s_node, s_val, rec, bd, s_acc, S); break;
        case 4: unit_eval<4, LUMP>(s_node, s_val, rec, bd, s_acc, S); break;
        case 3: unit_eval<3, LUMP>(s_node, s_val, rec, bd, s_acc, S); break;
        case 2: unit_eval<2, LUMP>(s_node, s_val, rec, bd, s_acc, S); break;
        case 1: unit_eval<1, LUMP>(s_node, s_val, rec, bd, s_acc, S); break;
        default: break;                  // pad unit (m = 0): no element
    }
}

// The chunk's fixed-point scale S = 2^(47 - e) and 1/S (as a pair), with
// B = 4 n_star Dmax vmax < 2^e: e from the binary exponents of Dmax and vmax
// and that of the product of their mantissas with 4 n_star (raised by a
// relative 2^-20, more than the two roundings of that product can lower
// it).  S = 0 when Dmax or vmax is 0 (no free node or every input 0: nothing
// to add) or not finite.  Every thread of the block computes the same pair.
__device__ __forceinline__ float2 unit_scale(float dmax, float vmax, int n_star) {
    if (!(dmax > 0.f) || !(vmax > 0.f) || !isfinite(dmax) || !isfinite(vmax)) return make_float2(0.f, 1.f);
    int ed, ev, ep;
    const float md = frexpf(dmax, &ed), mv = frexpf(vmax, &ev);     // mantissas in [0.5, 1)
    frexpf(md * mv * (4.0f * (float)n_star) * (1.0f + 0x1p-20f), &ep);
    const int e = max(-60, min(180, ed + ev + ep));
    const int sx = 47 - e;
    return make_float2(ldexpf(1.0f, max(-126, min(127, sx))), ldexpf(1.0f, max(-126, min(127, -sx))));
}

// Resident 128-thread blocks per SM the operator kernels are compiled for: it
// sets the register budget of a thread (65536 / (128 * 5) -> 96 registers,
// a few bytes of spills) and, with ~45 KB of shared memory per 3,072-tet
// chunk, five blocks (20 warps) fit an SM.  Measured on 160^3 Kuhn (one
// chunk per block): 169.7 us per pass against 175.1 us with four blocks (128
// registers), 193 us with three and 243 us with two.
constexpr int kUnitBlocks128 = 5;

// ---------------------------------------------------------------- phases of a chunk
struct UnitShared {
    NodeF *node;
    float *val;
    int *acc;          // two ints per node
    uint32_t *urec;    // the chunk's unit records
    float2 *ubd;       // beta*dt^2/6 per (element, half)
    uint64_t *bar;
};
__device__ __forceinline__ UnitShared unit_shared(unsigned char *smem, const UnitSmem &L) {
    UnitShared S;
    S.node = reinterpret_cast<NodeF *>(smem + L.node);
    S.val = reinterpret_cast<float *>(smem + L.val);
    S.acc = reinterpret_cast<int *>(smem + L.acc);
    S.urec = reinterpret_cast<uint32_t *>(smem + L.urec);
    S.ubd = reinterpret_cast<float2 *>(smem + L.ubd);
    S.bar = reinterpret_cast<uint64_t *>(smem + L.bar);
    return S;
}

// The fields of a chunk the paired kernels use (ChunkDesc, ChunkUnits).
struct UnitChunk {
    int node_off, n_loc, n_int, int_begin, sh_off, n_sh, unit_off, n_unit, max_star;
};
__device__ __forceinline__ UnitChunk unit_chunk(const MeshDev &m, int c) {
    const ChunkDesc cd = m.chunks[c];
    const ChunkUnits cu = m.chunks_u[c];
    return UnitChunk{cd.node_off, cd.n_loc, cd.n_int, cd.int_begin, cd.sh_off, cd.n_sh,
                     cu.unit_off, cu.n_unit, cu.max_star};
}

// One thread: bulk copies of the chunk's node records, shared-node
// destinations (into shd) and unit records with their beta*dt^2/6 (even unit
// counts: 16-byte multiples), all on one mbarrier phase.  Issued once per
// block, before any generic access of these buffers (no proxy fence).
__device__ __forceinline__ void unit_stage(const MeshDev &m, const UnitChunk &cd, const UnitShared &S,
                                           int32_t *shd) {
    const UnitChunk &cu = cd;
    const uint32_t b_node = (uint32_t)cd.n_loc * sizeof(NodeF);
    const uint32_t b_shd = (uint32_t)((cd.n_sh + kShPad - 1) / kShPad * kShPad) * 4u;
    const uint32_t b_rec = (uint32_t)cu.n_unit * kURecWords * 4u;
    const uint32_t b_bd = (uint32_t)cu.n_unit * kPatchMax * 8u;
    mbar_arrive_expect_tx(S.bar, b_node + b_shd + b_rec + b_bd);
    bulk_g2s(S.node, m.node32 + cd.node_off, b_node, S.bar);
    if (b_shd) bulk_g2s(shd, m.sh_dest + cd.sh_off, b_shd, S.bar);
    if (b_rec) {
        bulk_g2s(S.urec, m.urec + (int64_t)cu.unit_off * kURecWords, b_rec, S.bar);
        bulk_g2s(S.ubd, m.ubd + (int64_t)cu.unit_off * kPatchMax * 2, b_bd, S.bar);
    }
}

// p = D^-1 r + beta p on the chunk's nodes into val, node sums zeroed, the
// chunk maximum of |v| into *vmax.  Thread tid handles local nodes
// l = tid + NT j, up to eight per round, all loads of a round before any
// store (the stores to p could alias them): one round of loads for chunks of
// up to 8 NT nodes.  No Dirichlet mask is needed for v (D^-1 = 0 and r = 0
// there and p starts at 0).  Bit j of the result flags an interior Dirichlet
// node, D^-1 = 0 (its row of q is masked in the node phase; shared rows are
// masked by the update kernel).  Requires n_loc <= 32 NT.
template <int NT>
__device__ __forceinline__ uint32_t unit_gather(const Cg2Args<float> &a, const UnitChunk &cd, float beta,
                                                const UnitShared &S, unsigned int *vmax_out, int tid) {
    constexpr int kG = 8;
    const int n_loc = cd.n_loc, n_int = cd.n_int;
    float vmax = 0.f;
    uint32_t dmask = 0u;
    for (int l0 = tid, j0 = 0; l0 < n_loc; l0 += kG * NT, j0 += kG) {
        // interior nodes: D^-1, r, p contiguous from int_begin; shared
        // nodes: (D^-1 r, p) from the chunk's contiguous halo slots
        float dv[kG], rv[kG], pv[kG];
#pragma unroll
        for (int k = 0; k < kG; ++k) {
            const int l = l0 + k * NT;
            dv[k] = rv[k] = pv[k] = 0.f;
            if (l < n_int) {
                const int g = cd.int_begin + l;
                dv[k] = __ldg(a.dinv + g);
                rv[k] = a.r[g];
                pv[k] = a.p[g];
            } else if (l < n_loc) {
                const float2 h = a.halo[cd.sh_off + (l - n_int)];
                dv[k] = 1.f;
                rv[k] = h.x;
                pv[k] = h.y;
            }
        }
#pragma unroll
        for (int k = 0; k < kG; ++k) {
            const int l = l0 + k * NT;
            if (l < n_loc) {
                // shared nodes: fma(beta, p, 1 * z) = fma(beta, p, z), the value K2 stores
                const float v = cg_dir(dv[k], rv[k], beta, pv[k]);
                S.val[l] = v;
                reinterpret_cast<int2 *>(S.acc)[l] = make_int2(0, 0);
                vmax = fmaxf(vmax, fabsf(v));
                if (l < n_int) {
                    a.p[cd.int_begin + l] = v;
                    if (dv[k] == 0.f) dmask |= 1u << (j0 + k);
                }
            }
        }
    }
    // non-negative floats order as their bit patterns
    const unsigned int wmax = __reduce_max_sync(0xffffffffu, __float_as_uint(vmax));
    if ((tid & 31) == 0 && wmax) atomicMax(vmax_out, wmax);
    return dmask;
}

// Element phase: one unit per thread and round into the node sums (nothing
// to add when the scale is 0, i.e. every input is 0).
template <bool LUMP, int NT>
__device__ __forceinline__ void unit_elements(const UnitChunk &cu, const UnitShared &S, float scale, int tid) {
    if (scale == 0.f) return;
    for (int u = tid; u < cu.n_unit; u += NT) {
        const uint32_t *rec = S.urec + u * kURecWords;
        const float2 Su = make_float2(scale, (rec[0] & kUnitDup) ? 0.f : scale);
        unit_eval_any<LUMP>(S.node, S.val, rec, S.ubd + u * kPatchMax, S.acc, Su);
    }
}

// Node phase: each node's sum rounded to FP32 once, into q (interior, masked
// on Dirichlet rows) or the node's partial slot (shared); the thread's share
// of p.Ap = sum_e p_e^T A_e p_e over the chunk is returned.
template <int NT>
__device__ __forceinline__ DotF unit_nodes(const Cg2Args<float> &a, const UnitChunk &cd, const UnitShared &S,
                                           const int32_t *shd, float inv, uint32_t dmask, int tid) {
    DotF acc;
    for (int l = tid, j = 0; l < cd.n_loc; l += NT, ++j) {
        const int2 hl = reinterpret_cast<const int2 *>(S.acc)[l];
        float s = fmaf((float)hl.x, 16777216.0f, (float)hl.y) * inv;
        acc.add_prod(S.val[l], s);
        if (l < cd.n_int)
            a.q[cd.int_begin + l] = (dmask >> j) & 1u ? 0.f : s;
        else
            a.partial[shd[l - cd.n_int]] = s;
    }
    return acc;
}

// A chunk share not yet written: both words all ones (a NaN that no
// arithmetic produces; computed NaNs are 0x7fffffff).
__device__ __forceinline__ bool unit_unset(float v) { return __float_as_uint(v) == 0xffffffffu; }

// The operator pass's completion, in one extra block launched after the
// chunk blocks: each chunk block stores its share of p.Ap over the share's
// "unset" pattern and exits (no fence, no counter, no wait).  This block
// polls the shares in chunk order until each is set (bounded), sums them in
// a fixed order and sets alpha = rz / p.Ap, and restores the unset pattern
// for the next launch.  The chunk blocks never wait for it, so they always
// complete; on timeout the error flag is set, alpha is left unchanged and
// the shares are reset all the same (and again, on the stream, at the start
// of the next CG run, in case a late chunk block wrote its share after).
template <int NT>
__device__ __noinline__ void unit_reduce_alpha(const Cg2Args<float> &a, int n_chunks, int *err, int tid) {
    __shared__ float2 s_w[NT / 32];
    // eight 16-byte loads (two chunk shares each) in flight per thread:
    // thread t takes the chunk pairs j = t + NT (8 i + k), chunks 2j and
    // 2j + 1, into accumulator k, merged in k order (the share array holds
    // at least one entry past the last chunk, so the pair load stays inside)
    constexpr int kAcc = 8;
    DotF part[kAcc];
    float4 *pq4 = reinterpret_cast<float4 *>(a.pq);
    const int n_pairs = (n_chunks + 1) / 2;
    uint32_t polls = 0;
    bool ok = true;
    for (int j0 = tid; j0 < n_pairs; j0 += NT * kAcc) {
        float4 v[kAcc];
#pragma unroll
        for (int k = 0; k < kAcc; ++k) {
            const int j = j0 + NT * k;
            v[k] = j < n_pairs ? __ldcg(pq4 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < kAcc; ++k) {
            const int j = j0 + NT * k;
            if (j >= n_pairs) continue;
            const bool two = 2 * j + 1 < n_chunks;
            // wait (bounded) for the shares of chunks 2j and 2j + 1
            while (ok && (unit_unset(v[k].x) || unit_unset(v[k].y) ||
                          (two && (unit_unset(v[k].z) || unit_unset(v[k].w))))) {
                if (++polls > kGridSpinLimit) {
                    ok = false;
                    break;
                }
                __nanosleep(64);
                v[k] = __ldcg(pq4 + j);
            }
            part[k].merge(v[k].x, v[k].y);
            if (two) part[k].merge(v[k].z, v[k].w);
        }
        if (!ok) break;
    }
    ok = __syncthreads_and(ok);   // every share read
    for (int j = tid; j < n_pairs; j += NT)
        __stcg(pq4 + j, make_float4(__uint_as_float(0xffffffffu), __uint_as_float(0xffffffffu),
                                    __uint_as_float(0xffffffffu), __uint_as_float(0xffffffffu)));
    if (!ok) {
        if (tid == 0) atomicOr(err, kErrGridTimeout);
        return;
    }
    DotF acc = part[0];
#pragma unroll
    for (int k = 1; k < kAcc; ++k) acc.merge(part[k].hi, part[k].lo);
    acc = warp_merge(acc);
    if ((tid & 31) == 0) s_w[tid >> 5] = make_float2(acc.hi, acc.lo);
    __syncthreads();
    if (tid == 0) {
        DotF t;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) t.merge(s_w[w].x, s_w[w].y);
        const double pq = (double)t.hi + (double)t.lo;
        CgState *st = a.st;
        st->pq = pq;
        if (!(pq > 0.0) || !isfinite(pq)) {
            st->status = kCgBreakdown;
            st->done = 1;
        } else {
            st->alpha = st->rz / pq;
        }
    }
}

// The chunk's share of p.Ap from the threads' accumulators: each warp merges
// its lanes (fixed tree), warp w writes wdot[w]; after a barrier one thread
// merges the warps in order (chunk_share).
template <int NT>
__device__ __forceinline__ void unit_warp_share(DotF acc, float2 *wdot, int tid) {
    acc = warp_merge(acc);
    if ((tid & 31) == 0) wdot[tid >> 5] = make_float2(acc.hi, acc.lo);
}
template <int NT>
__device__ __forceinline__ float2 chunk_share(const float2 *wdot) {
    DotF t;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) t.merge(wdot[w].x, wdot[w].y);
    return part_pack((double)t.hi + (double)t.lo);
}

// K1 on paired patches: one block of NT threads (128 or 256) per chunk and
// one more block (the last) for the completion, MINB blocks per SM (the
// register budget of a thread).
template <bool LUMP, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_cg2_units(MeshDev m, Cg2Args<float> a) {
    extern __shared__ __align__(128) unsigned char smem[];
    const UnitShared S = unit_shared(smem, m.smu);
    int32_t *s_shd = reinterpret_cast<int32_t *>(smem + m.smu.shd);
    __shared__ float s_beta;
    __shared__ unsigned int s_vmax;
    __shared__ int s_done;
    __shared__ float2 s_wdot[NT / 32];
    __shared__ UnitChunk s_uc;
    const int tid = threadIdx.x;
    if (blockIdx.x == (unsigned)m.n_chunks) {
        if (tid == 0) s_done = ld_flag(&a.st->done);
        __syncthreads();
        if (!s_done) unit_reduce_alpha<NT>(a, m.n_chunks, m.err, tid);
        return;
    }
    // the chunk's fields: in registers for the staging and the gather (read
    // together with the CG state), from shared memory in the later phases
    const UnitChunk uc = unit_chunk(m, blockIdx.x);
    if (tid == 0) {
        s_done = a.st->done;
        s_beta = (float)a.st->beta;
        s_vmax = 0u;
        s_uc = uc;
        mbar_init(S.bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (s_done) return;
    if (tid == 0) unit_stage(m, uc, S, s_shd);
    const uint32_t dmask = unit_gather<NT>(a, uc, s_beta, S, &s_vmax, tid);
    const float dmax = __ldg(m.dmax + blockIdx.x);
    {
        bool ok = mbar_wait_bounded(S.bar, 0);
        ok = __syncthreads_and(ok);   // also publishes val, acc and s_vmax
        if (!ok) {
            if (tid == 0) atomicOr(m.err, kErrMbarTimeout);
            mbar_wait_bounded(S.bar, 0);
            return;
        }
    }
    const float2 sc = unit_scale(dmax, __uint_as_float(s_vmax), s_uc.max_star);
    unit_elements<LUMP, NT>(s_uc, S, sc.x, tid);
    __syncthreads();
    unit_warp_share<NT>(unit_nodes<NT>(a, s_uc, S, s_shd, sc.y, dmask, tid), s_wdot, tid);
    __syncthreads();
    if (tid == 0) a.pq[blockIdx.x] = chunk_share<NT>(s_wdot);   // one 8-byte store over the unset pattern
}

// Largest diagonal entry D_jj = 1 / D^-1_jj over each chunk's free local nodes
// (the fixed-point bound of k_cg2_units); one block per chunk, after every
// diagonal update.
static __global__ void k_chunk_dmax(MeshDev m, float *__restrict__ dmax) {
    const ChunkDesc cd = m.chunks[blockIdx.x];
    float mx = 0.f;
    for (int l = threadIdx.x; l < cd.n_loc; l += blockDim.x) {
        const int g = l < cd.n_int ? cd.int_begin + l : m.sh_ids[cd.sh_off + (l - cd.n_int)];
        const float di = m.dinv32[g];
        if (di > 0.f) mx = fmaxf(mx, 1.0f / di);
    }
    const unsigned int wmax = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
    __shared__ unsigned int s_mx;
    if (threadIdx.x == 0) s_mx = 0u;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) atomicMax(&s_mx, wmax);
    __syncthreads();
    // a little above the FP32 value: the bound must hold for the exact D
    if (threadIdx.x == 0) dmax[blockIdx.x] = __uint_as_float(s_mx) * 1.0001f;
}

// The halo of the paired-patch kernel: every chunk-major shared slot j (node
// i = sh_ids[j]) gets (D^-1_i r_i, p_i) -- after each update kernel (the next
// operator pass reads it contiguously per chunk), at the start of a CG run
// and before ps_debug_cg_apply.  Pads (sh_ids = -1) are skipped.  Inside the
// iteration (reduce = 1) the first block instead sums the update kernel's
// block shares of rz and rr in block order and ends the iteration
// (cg2_update_tail), while the other blocks gather; a run that was already
// done before this iteration's update kernel does nothing.
static __global__ void __launch_bounds__(256) k_halo_gather(int64_t n_slots, const int32_t *__restrict__ sh_ids,
                                                            Cg2Args<float> a, int reduce) {
    if (reduce) {
        if (ld_flag(&a.st->done)) return;
        if (blockIdx.x == 0) {
            __shared__ double red[34];
            double rz, rr;
            part_sum2(a.z2, a.z2 + a.g3, a.g3, red, rz, rr);
            if (threadIdx.x == 0) cg2_update_tail(a.st, rz, rr);
            return;
        }
    }
    const int64_t b = reduce ? blockIdx.x - 1 : blockIdx.x, nb = reduce ? gridDim.x - 1 : gridDim.x;
    const float *__restrict__ r = a.r;
    const float *__restrict__ p = a.p;
    const float *__restrict__ dinv = a.dinv;
    for (int64_t j = b * blockDim.x + threadIdx.x; j < n_slots; j += nb * blockDim.x) {
        const int i = __ldg(sh_ids + j);
        if (i >= 0) a.halo[j] = make_float2(__fmul_rn(__ldg(dinv + i), r[i]), p[i]);
    }
}

// beta*dt^2/6 of every (unit, element, half) slot from the caller's beta
// (0 on slots without an element).
static __global__ void k_set_beta_units(int64_t n, const int32_t *__restrict__ uelem, const double *__restrict__ beta,
                                        double dt2, float *__restrict__ ubd) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int e = uelem[k];
        ubd[k] = e >= 0 ? (float)(beta[e] * dt2 * (1.0 / 6.0)) : 0.f;
    }
}

}  // namespace ps
