// Host preprocessing: Morton chunking, node renumbering, local connectivity.
// See layout.h for the layout this produces.
#include "mesh_prep.h"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>

namespace ps {

namespace {

// Spread the low 21 bits of v so that they occupy every third bit.
inline uint64_t spread3(uint64_t v) {
    v &= 0x1fffffULL;
    v = (v | (v << 32)) & 0x1f00000000ffffULL;
    v = (v | (v << 16)) & 0x1f0000ff0000ffULL;
    v = (v | (v << 8)) & 0x100f00f00f00f00fULL;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ULL;
    v = (v | (v << 2)) & 0x1249249249249249ULL;
    return v;
}

// Spread the low 31 bits of v so that they occupy every second bit.
inline uint64_t spread2(uint64_t v) {
    v &= 0x7fffffffULL;
    v = (v | (v << 16)) & 0x0000ffff0000ffffULL;
    v = (v | (v << 8)) & 0x00ff00ff00ff00ffULL;
    v = (v | (v << 4)) & 0x0f0f0f0f0f0f0f0fULL;
    v = (v | (v << 2)) & 0x3333333333333333ULL;
    v = (v | (v << 1)) & 0x5555555555555555ULL;
    return v;
}

// Stable LSD radix sort of (key, id) by key, 16-bit digits.
void radix_sort(std::vector<uint64_t> &key, std::vector<int32_t> &id) {
    const size_t n = key.size();
    std::vector<uint64_t> k2(n);
    std::vector<int32_t> i2(n);
    std::vector<size_t> cnt(65537);
    uint64_t all = 0;
    for (uint64_t k : key) all |= k;
    for (int shift = 0; shift < 64; shift += 16) {
        if (((all >> shift) & 0xffffULL) == 0) continue;
        std::fill(cnt.begin(), cnt.end(), 0);
        for (size_t i = 0; i < n; ++i) cnt[((key[i] >> shift) & 0xffff) + 1]++;
        for (int b = 0; b < 65536; ++b) cnt[b + 1] += cnt[b];
        for (size_t i = 0; i < n; ++i) {
            size_t d = cnt[(key[i] >> shift) & 0xffff]++;
            k2[d] = key[i];
            i2[d] = id[i];
        }
        key.swap(k2);
        id.swap(i2);
    }
}

double simplex_det(int dim, const double *coords, const int32_t *v) {
    if (dim == 2) {
        const double *a = coords + 2 * (int64_t)v[0], *b = coords + 2 * (int64_t)v[1],
                     *c = coords + 2 * (int64_t)v[2];
        return (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]);
    }
    const double *a = coords + 3 * (int64_t)v[0];
    double e[3][3];
    for (int k = 0; k < 3; ++k) {
        const double *p = coords + 3 * (int64_t)v[k + 1];
        for (int c = 0; c < 3; ++c) e[k][c] = p[c] - a[c];
    }
    return e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
           e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
           e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
}

// One star patch under construction (chunk-local ids).
struct PatchRec {
    int m = 0;
    int a = 0, b = 0;
    int ring[kPatchMax + 1];
    int elem[kPatchMax];   // chunk-local element index
};

// Group the elements of one chunk into star patches.  lc: [n][4] local vertex
// ids; lx: [local node][dim] coordinates (3D only, may be null).  Pivots are
// edges (3D) or vertices (2D); pivots are taken greedily by the number of
// still unassigned elements around them (more first; among equal counts the
// longer edge first, then by pivot key), and the unassigned elements around a
// pivot are linked into chains through their shared ring vertices, at most
// kPatchMax per chain.  Whatever is left becomes patches of one element.
// Longer edges first: on Kuhn-type meshes the six tetrahedra of a cube cell
// share its main diagonal, the longest edge of the cell, so every cell
// becomes one closed star of six.
void build_patches(int dim, int n, const std::vector<std::array<int, 4>> &lc, std::vector<PatchRec> &out,
                   const double *lx) {
    const int nv = dim + 1;
    out.clear();
    std::vector<char> used(n, 0);
    std::vector<std::pair<uint64_t, int>> inc;   // (pivot key, element)
    inc.reserve((size_t)n * (dim == 3 ? 6 : 3));
    for (int e = 0; e < n; ++e) {
        if (dim == 3) {
            for (int i = 0; i < 4; ++i)
                for (int j = i + 1; j < 4; ++j) {
                    uint64_t u = (uint64_t)std::min(lc[e][i], lc[e][j]);
                    uint64_t v = (uint64_t)std::max(lc[e][i], lc[e][j]);
                    inc.push_back({(u << 20) | v, e});
                }
        } else {
            for (int i = 0; i < 3; ++i) inc.push_back({(uint64_t)lc[e][i], e});
        }
    }
    std::sort(inc.begin(), inc.end());
    std::vector<size_t> gstart;
    for (size_t k = 0; k < inc.size(); ++k)
        if (k == 0 || inc[k].first != inc[k - 1].first) gstart.push_back(k);
    gstart.push_back(inc.size());
    const size_t ng = gstart.size() - 1;
    int maxc = 0;
    for (size_t g = 0; g < ng; ++g) maxc = std::max(maxc, (int)(gstart[g + 1] - gstart[g]));
    // visiting order of the pivots: longer edges first (3D with coordinates),
    // ties by pivot key
    std::vector<size_t> gorder(ng);
    for (size_t g = 0; g < ng; ++g) gorder[g] = g;
    if (dim == 3 && lx) {
        std::vector<double> len2(ng);
        for (size_t g = 0; g < ng; ++g) {
            const uint64_t key = inc[gstart[g]].first;
            const int u = (int)(key >> 20), v = (int)(key & 0xfffff);
            double s2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                const double d = lx[(size_t)u * 3 + k] - lx[(size_t)v * 3 + k];
                s2 += d * d;
            }
            len2[g] = s2;
        }
        std::stable_sort(gorder.begin(), gorder.end(), [&](size_t x, size_t y) { return len2[x] > len2[y]; });
    }
    std::vector<int> cand;
    std::vector<std::array<int, 2>> rp;   // ring pair of each candidate
    for (int c = maxc; c >= 2; --c) {
        for (size_t gi = 0; gi < ng; ++gi) {
            const size_t g = gorder[gi];
            cand.clear();
            for (size_t k = gstart[g]; k < gstart[g + 1]; ++k)
                if (!used[inc[k].second]) cand.push_back(inc[k].second);
            if ((int)cand.size() < c) continue;
            const uint64_t key = inc[gstart[g]].first;
            int pa, pb = 0;
            if (dim == 3) {
                pa = (int)(key >> 20);
                pb = (int)(key & 0xfffff);
            } else {
                pa = (int)key;
            }
            rp.clear();
            for (int e : cand) {
                std::array<int, 2> r{-1, -1};
                int t = 0;
                for (int i = 0; i < nv; ++i) {
                    int v = lc[e][i];
                    if (v == pa || (dim == 3 && v == pb)) continue;
                    if (t < 2) r[t++] = v;
                }
                rp.push_back(r);
            }
            std::vector<char> taken(cand.size(), 0);
            size_t left = cand.size();
            while (left > 0) {
                // start from a ring vertex of degree 1 among the remaining, if any
                int start = -1;
                for (size_t i = 0; i < cand.size() && start < 0; ++i) {
                    if (taken[i]) continue;
                    for (int s2 = 0; s2 < 2 && start < 0; ++s2) {
                        int v = rp[i][s2], deg = 0;
                        for (size_t k = 0; k < cand.size(); ++k)
                            if (!taken[k] && (rp[k][0] == v || rp[k][1] == v)) ++deg;
                        if (deg == 1) start = v;
                    }
                }
                if (start < 0)
                    for (size_t i = 0; i < cand.size(); ++i)
                        if (!taken[i]) { start = rp[i][0]; break; }
                PatchRec P;
                P.a = pa;
                P.b = pb;
                P.ring[0] = start;
                int cur = start;
                while (P.m < kPatchMax) {
                    int pick = -1;
                    for (size_t k = 0; k < cand.size(); ++k)
                        if (!taken[k] && (rp[k][0] == cur || rp[k][1] == cur)) { pick = (int)k; break; }
                    if (pick < 0) break;
                    taken[pick] = 1;
                    --left;
                    int nxt = rp[pick][0] == cur ? rp[pick][1] : rp[pick][0];
                    P.elem[P.m] = cand[pick];
                    P.ring[P.m + 1] = nxt;
                    ++P.m;
                    cur = nxt;
                }
                if (P.m == 0) break;   // cannot happen: start has an element
                for (int j = 0; j < P.m; ++j) used[P.elem[j]] = 1;
                out.push_back(P);
            }
        }
    }
    for (int e = 0; e < n; ++e) {
        if (used[e]) continue;
        PatchRec P;
        P.m = 1;
        P.a = lc[e][0];
        if (dim == 3) {
            P.b = lc[e][1];
            P.ring[0] = lc[e][2];
            P.ring[1] = lc[e][3];
        } else {
            P.b = 0;
            P.ring[0] = lc[e][1];
            P.ring[1] = lc[e][2];
        }
        P.elem[0] = e;
        out.push_back(P);
    }
}

}  // namespace

// Order the patches of a chunk for the kernels' assignment (patch q is
// evaluated by thread q mod kChunkThreads, in round q / kChunkThreads): largest
// patches first, every other round reversed, so that the element counts of
// the threads of a block are close and the block waits less at the barrier
// that ends the element phase.
static void balance_patches(std::vector<PatchRec> &p) {
    std::stable_sort(p.begin(), p.end(), [](const PatchRec &x, const PatchRec &y) { return x.m > y.m; });
    for (size_t r = 1; r * kChunkThreads < p.size(); r += 2) {
        const size_t b = r * kChunkThreads, e = std::min(p.size(), b + kChunkThreads);
        std::reverse(p.begin() + b, p.begin() + e);
    }
}

std::string prepare_mesh(int dim, int64_t n_nodes, const double *coords, int64_t n_elems,
                         const int32_t *conn, const uint8_t *dirichlet, const PrepOptions &opt,
                         PrepMesh &m) {
    if (dim != 2 && dim != 3) return "dim must be 2 or 3";
    if (n_nodes < 1 || n_elems < 1) return "empty mesh";
    if (n_nodes >= (int64_t)INT32_MAX || n_elems >= (int64_t)INT32_MAX / 4) return "mesh too large";
    const int nv = dim + 1;
    m = PrepMesh();
    m.dim = dim;
    m.nv = nv;
    m.n_nodes = n_nodes;
    m.n_elems = n_elems;

    // ---- validation
    for (int64_t i = 0; i < n_nodes * dim; ++i)
        if (!std::isfinite(coords[i])) return "non-finite coordinate";
    for (int64_t i = 0; i < n_elems * nv; ++i)
        if (conn[i] < 0 || conn[i] >= n_nodes) return "vertex id out of range";
    // periodic merging: every vertex's master (itself without merging)
    std::vector<int32_t> master(n_nodes);
    for (int64_t i = 0; i < n_nodes; ++i) master[i] = (int32_t)i;
    if (opt.periodic) {
        for (int64_t i = 0; i < n_nodes; ++i) {
            const int32_t mi = opt.periodic[i];
            if (mi < 0 || mi >= n_nodes) return "periodic master out of range";
            if (opt.periodic[mi] != mi) return "periodic master is itself merged into another vertex";
            if (dirichlet && (dirichlet[i] != 0) != (dirichlet[mi] != 0))
                return "periodic vertex and its master differ in the Dirichlet flag";
            master[i] = mi;
        }
        for (int64_t e = 0; e < n_elems; ++e)
            for (int a = 0; a < nv; ++a)
                for (int b = a + 1; b < nv; ++b)
                    if (master[conn[e * nv + a]] == master[conn[e * nv + b]])
                        return "element with two vertices merged into one unknown";
    }
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int c = 0; c < dim; ++c) lo[c] = hi[c] = coords[c];
    for (int64_t i = 0; i < n_nodes; ++i)
        for (int c = 0; c < dim; ++c) {
            lo[c] = std::min(lo[c], coords[i * dim + c]);
            hi[c] = std::max(hi[c], coords[i * dim + c]);
        }
    double ext = 0;
    for (int c = 0; c < dim; ++c) ext = std::max(ext, hi[c] - lo[c]);
    if (!(ext > 0)) return "degenerate bounding box";
    const double vol_floor = std::pow(ext, dim) * 1e-30;
    double det_sum = 0.0;
    for (int64_t e = 0; e < n_elems; ++e) {
        double d = simplex_det(dim, coords, conn + e * nv);
        if (!(std::fabs(d) > vol_floor)) return "element of zero volume";
        det_sum += std::fabs(d);
        for (int a = 0; a < nv; ++a)
            for (int b = a + 1; b < nv; ++b)
                if (conn[e * nv + a] == conn[e * nv + b]) return "repeated vertex in element";
    }

    // ---- Morton order of element centroids
    // The quantum is a power-of-two fraction of the typical cell size
    // h = (mean |det|)^(1/d) (the edge of the cube that d! mean elements
    // fill), so that on structured (Kuhn-type) meshes every cell maps to one
    // key prefix and aligned Morton blocks are blocks of whole cells, whatever
    // the number of cells per side.
    std::vector<uint64_t> key(n_elems);
    std::vector<int32_t> order(n_elems);
    const int bits = dim == 3 ? 21 : 31;
    const double qmax = (double)((1ULL << bits) - 1);
    const double h = std::pow(det_sum / (double)n_elems, 1.0 / dim);
    double scale = qmax / ext;
    if (h > 0 && std::isfinite(h)) {
        const int s = (int)std::floor(std::log2(qmax * h / ext));
        if (s >= 0) scale = std::ldexp(1.0, s) / h;
    }
    for (int64_t e = 0; e < n_elems; ++e) {
        double cen[3] = {0, 0, 0};
        for (int a = 0; a < nv; ++a)
            for (int c = 0; c < dim; ++c) cen[c] += coords[(int64_t)conn[e * nv + a] * dim + c];
        uint64_t q[3] = {0, 0, 0};
        for (int c = 0; c < dim; ++c) {
            double t = (cen[c] / nv - lo[c]) * scale;
            t = std::min(std::max(t, 0.0), (double)((1ULL << bits) - 1));
            q[c] = (uint64_t)t;
        }
        key[e] = dim == 3 ? (spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2))
                          : (spread2(q[0]) | (spread2(q[1]) << 1));
        order[e] = (int32_t)e;
    }
    radix_sort(key, order);
    key.clear();
    key.shrink_to_fit();

    // ---- chunk sizes
    int ec = opt.chunk_elems;
    if (ec <= 0) {
        // aim for >= 4 chunks per SM of a 152-SM part, 96..1536 elements each
        int64_t t = n_elems / 608;
        t = std::max<int64_t>(96, std::min<int64_t>(1536, t));
        if (dim == 3) {
            // 6 * 2^k tets: on Kuhn-type meshes (6 tets per cube cell) such a
            // chunk is a Morton block of cells, with the fewest shared nodes
            int64_t b = 96;
            while (b < t && b < 1536) b *= 2;
            t = b;
            // large meshes: 8^3-cell blocks; fewer shared nodes outweigh the
            // lower occupancy of the larger shared-memory footprint once
            // there are many waves of chunks (measured on 128^3: -14% per pass)
            if (n_elems >= (int64_t)3072 * 152 * 8) t = 3072;
        }
        ec = (int)round_up(t, 32);
    }
    ec = std::max(1, std::min(ec, kMaxChunkPatches));
    int nmax = opt.chunk_nodes_max > 0 ? opt.chunk_nodes_max : std::max(ec, nv * 64);
    nmax = std::max(nmax, nv);
    nmax = std::min(nmax, 65535);

    // ---- greedy chunking along the Morton order
    std::vector<int32_t> stamp(n_nodes, -1);
    std::vector<int64_t> chunk_begin;   // index into `order`
    {
        int64_t cur_e = 0;
        int cur_n = 0, cid = 0;
        chunk_begin.push_back(0);
        for (int64_t k = 0; k < n_elems; ++k) {
            const int32_t *v = conn + (int64_t)order[k] * nv;
            int add = 0;
            for (int a = 0; a < nv; ++a) add += stamp[v[a]] != cid;
            if (cur_e > 0 && (cur_e >= ec || cur_n + add > nmax)) {
                ++cid;
                chunk_begin.push_back(k);
                cur_e = 0;
                cur_n = 0;
                add = nv;
            }
            for (int a = 0; a < nv; ++a)
                if (stamp[v[a]] != cid) { stamp[v[a]] = cid; }
            cur_n += add;
            ++cur_e;
        }
        chunk_begin.push_back(n_elems);
    }
    if (opt.split_lead > 0 && (int64_t)chunk_begin.size() - 1 >= 4 * (int64_t)opt.split_lead) {
        // the first split_lead chunks in two halves each (each half is
        // contiguous in the Morton order: on Kuhn meshes a block of cells)
        std::vector<int64_t> nb;
        nb.reserve(chunk_begin.size() + opt.split_lead);
        for (size_t c = 0; c + 1 < chunk_begin.size(); ++c) {
            nb.push_back(chunk_begin[c]);
            if ((int)c < opt.split_lead && chunk_begin[c + 1] - chunk_begin[c] >= 2)
                nb.push_back((chunk_begin[c] + chunk_begin[c + 1]) / 2);
        }
        nb.push_back(n_elems);
        chunk_begin.swap(nb);
    }
    const int nc = (int)chunk_begin.size() - 1;
    m.n_chunks = nc;

    // ---- classify unknowns (by master vertex): interior = one vertex, touched
    // by one chunk; shared = touched by several chunks, or carrying merged
    // periodic vertices (each vertex keeps its own coordinates, so a merged
    // unknown gets one local node per vertex, summed like partials)
    std::vector<int32_t> last(n_nodes, -1);
    std::vector<uint8_t> shared(n_nodes, 0), used(n_nodes, 0);
    for (int64_t i = 0; i < n_nodes; ++i)
        if (master[i] != i) shared[master[i]] = 1;
    for (int c = 0; c < nc; ++c)
        for (int64_t k = chunk_begin[c]; k < chunk_begin[c + 1]; ++k) {
            const int32_t *v = conn + (int64_t)order[k] * nv;
            for (int a = 0; a < nv; ++a) {
                used[v[a]] = 1;
                const int32_t d = master[v[a]];
                if (last[d] != c) {
                    if (last[d] != -1) shared[d] = 1;
                    last[d] = c;
                }
            }
        }
    for (int64_t i = 0; i < n_nodes; ++i)
        if (!used[i]) return "node not used by any element";

    // ---- renumber unknowns: interior per chunk, then shared
    std::vector<int32_t> dof(n_nodes, -1);   // new id of each master vertex
    m.chunks.resize(nc);
    int32_t next = 0;
    for (int c = 0; c < nc; ++c) {
        ChunkDesc &cd = m.chunks[c];
        std::memset(&cd, 0, sizeof(cd));
        cd.int_begin = next;
        for (int64_t k = chunk_begin[c]; k < chunk_begin[c + 1]; ++k) {
            const int32_t *v = conn + (int64_t)order[k] * nv;
            for (int a = 0; a < nv; ++a) {
                const int32_t d = master[v[a]];
                if (!shared[d] && dof[d] < 0) dof[d] = next++;
            }
        }
        cd.n_int = next - cd.int_begin;
    }
    m.n_int = next;
    for (int c = 0; c < nc; ++c)
        for (int64_t k = chunk_begin[c]; k < chunk_begin[c + 1]; ++k) {
            const int32_t *v = conn + (int64_t)order[k] * nv;
            for (int a = 0; a < nv; ++a) {
                const int32_t d = master[v[a]];
                if (shared[d] && dof[d] < 0) dof[d] = next++;
            }
        }
    m.n_shared = next - m.n_int;
    m.n_dofs = next;
    m.new_of_old.assign(n_nodes, -1);
    for (int64_t i = 0; i < n_nodes; ++i) m.new_of_old[i] = dof[master[i]];
    m.old_of_new.assign(m.n_dofs, 0);
    m.dirichlet_new.assign(m.n_dofs, 0);
    for (int64_t i = 0; i < n_nodes; ++i)
        if (master[i] == i) {
            m.old_of_new[dof[i]] = (int32_t)i;
            m.dirichlet_new[dof[i]] = dirichlet ? (dirichlet[i] != 0) : 0;
        }
    m.n_free = 0;
    for (int64_t g = 0; g < m.n_dofs; ++g) m.n_free += m.dirichlet_new[g] == 0;
    if (opt.periodic) {
        // merged vertices of every unknown, ascending vertex id
        m.slave_ptr.assign(m.n_dofs + 1, 0);
        for (int64_t i = 0; i < n_nodes; ++i)
            if (master[i] != i) m.slave_ptr[dof[master[i]] + 1]++;
        for (int64_t g = 0; g < m.n_dofs; ++g) m.slave_ptr[g + 1] += m.slave_ptr[g];
        m.slave.assign(m.slave_ptr.back(), 0);
        std::vector<int32_t> fill(m.slave_ptr.begin(), m.slave_ptr.end() - 1);
        for (int64_t i = 0; i < n_nodes; ++i)
            if (master[i] != i) m.slave[fill[dof[master[i]]]++] = (int32_t)i;
    }

    // ---- per-chunk local structure
    int64_t patch_off = 0, node_off = 0, sh_off = 0, incp_off = 0, inc_off = 0;
    std::vector<int32_t> loc_of_vtx(n_nodes, -1);   // local node of a vertex in the current chunk
    std::vector<int32_t> shl;                        // the chunk's shared local vertices
    std::vector<int32_t> shr_cnt(m.n_shared + 1, 0);
    std::vector<std::array<int, 4>> lc;
    std::vector<PatchRec> patches;
    std::vector<double> lxyz;                        // the chunk's local node coordinates (3D)
    for (int c = 0; c < nc; ++c) {
        ChunkDesc &cd = m.chunks[c];
        const int n_el = (int)(chunk_begin[c + 1] - chunk_begin[c]);
        cd.n_elem = n_el;
        // shared local nodes: one per vertex whose unknown is shared,
        // ascending (unknown, vertex)
        shl.clear();
        for (int64_t k = chunk_begin[c]; k < chunk_begin[c + 1]; ++k) {
            const int32_t *v = conn + (int64_t)order[k] * nv;
            for (int a = 0; a < nv; ++a) {
                const int32_t g = m.new_of_old[v[a]];
                if (g >= m.n_int && loc_of_vtx[v[a]] != -2) { loc_of_vtx[v[a]] = -2; shl.push_back(v[a]); }
            }
        }
        std::sort(shl.begin(), shl.end(), [&](int32_t x, int32_t y) {
            const int32_t gx = m.new_of_old[x], gy = m.new_of_old[y];
            return gx != gy ? gx < gy : x < y;
        });
        cd.n_sh = (int32_t)shl.size();
        cd.n_loc = cd.n_int + cd.n_sh;
        cd.node_off = (int32_t)node_off;
        cd.sh_off = (int32_t)sh_off;
        cd.incp_off = (int32_t)incp_off;
        for (int32_t l = 0; l < cd.n_int; ++l) loc_of_vtx[m.old_of_new[cd.int_begin + l]] = l;
        for (int32_t j = 0; j < cd.n_sh; ++j) {
            const int32_t g = m.new_of_old[shl[j]];
            loc_of_vtx[shl[j]] = cd.n_int + j;
            m.sh_ids.push_back(g);
            shr_cnt[g - m.n_int + 1]++;
        }
        for (int64_t j = cd.n_sh; j < round_up(cd.n_sh, kShPad); ++j) m.sh_ids.push_back(-1);
        sh_off += round_up(cd.n_sh, kShPad);
        node_off += cd.n_loc;
        // local connectivity and star patches
        lc.assign(n_el, std::array<int, 4>{0, 0, 0, 0});
        for (int e = 0; e < n_el; ++e) {
            int32_t src = order[chunk_begin[c] + e];
            for (int a = 0; a < nv; ++a) lc[e][a] = loc_of_vtx[conn[(int64_t)src * nv + a]];
        }
        if (dim == 3) {
            lxyz.resize((size_t)cd.n_loc * 3);
            for (int32_t l = 0; l < cd.n_loc; ++l) {
                const int32_t vtx = l < cd.n_int ? m.old_of_new[cd.int_begin + l] : shl[l - cd.n_int];
                for (int k = 0; k < 3; ++k) lxyz[(size_t)l * 3 + k] = coords[(int64_t)vtx * 3 + k];
            }
        }
        build_patches(dim, n_el, lc, patches, dim == 3 ? lxyz.data() : nullptr);
        balance_patches(patches);
        const int np = (int)patches.size();
        if (np > kMaxChunkPatches) return "internal: too many patches in a chunk";
        cd.patch_off = (int32_t)patch_off;
        cd.n_patch = np;
        const int64_t np_pad = round_up(np, kPatchPad);
        m.pids.resize((patch_off + np_pad) * kPatchIds, 0);
        m.elem_src.resize((patch_off + np_pad) * kPatchMax, -1);
        std::vector<int32_t> cnt(cd.n_loc + 1, 0);
        auto each_slot = [&](const PatchRec &P, auto &&fn) {
            fn(P.a, 0);
            if (dim == 3) fn(P.b, 1);
            for (int j = 0; j <= P.m; ++j) fn(P.ring[j], 2 + j);
        };
        for (int q = 0; q < np; ++q) {
            const PatchRec &P = patches[q];
            uint16_t *rec = &m.pids[(patch_off + q) * kPatchIds];
            rec[0] = (uint16_t)P.m;
            rec[1] = (uint16_t)P.a;
            rec[2] = (uint16_t)(dim == 3 ? P.b : P.a);
            for (int j = 0; j <= P.m; ++j) rec[3 + j] = (uint16_t)P.ring[j];
            for (int j = 0; j < P.m; ++j)
                m.elem_src[(patch_off + q) * kPatchMax + j] = order[chunk_begin[c] + P.elem[j]];
            each_slot(P, [&](int node, int) { cnt[node + 1]++; });
        }
        for (int32_t l = 0; l < cd.n_loc; ++l) cnt[l + 1] += cnt[l];
        const int n_inc = cnt[cd.n_loc];
        for (int32_t l = 0; l <= cd.n_loc; ++l) m.incp.push_back((uint16_t)cnt[l]);
        for (int64_t j = cd.n_loc + 1; j < round_up(cd.n_loc + 1, kIncpPad); ++j) m.incp.push_back((uint16_t)n_inc);
        incp_off += round_up(cd.n_loc + 1, kIncpPad);
        cd.inc_off = (int32_t)inc_off;
        cd.n_inc = n_inc;
        m.inc.resize(inc_off + round_up(n_inc, kIncPad), 0);
        {
            std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
            for (int q = 0; q < np; ++q)
                each_slot(patches[q], [&](int node, int slot) {
                    m.inc[inc_off + fill[node]++] = (uint16_t)(q * kPatchSlots + slot);
                });
        }
        inc_off += round_up(n_inc, kIncPad);
        patch_off += np_pad;
        m.n_patches += np;
        // node block bookkeeping (coordinates of each local node's own
        // vertex, relative to the chunk origin)
        const int32_t origin_vtx = cd.n_int > 0 ? m.old_of_new[cd.int_begin] : shl[0];
        const double *o = coords + (int64_t)origin_vtx * dim;
        for (int32_t l = 0; l < cd.n_loc; ++l) {
            const int32_t vtx = l < cd.n_int ? m.old_of_new[cd.int_begin + l] : shl[l - cd.n_int];
            m.loc_node.push_back(m.new_of_old[vtx]);
            m.loc_orig.push_back(vtx);
            const double *p = coords + (int64_t)vtx * dim;
            for (int k = 0; k < dim; ++k) m.loc_rel.push_back(p[k] - o[k]);
        }
        for (int32_t l = 0; l < cd.n_int; ++l) loc_of_vtx[m.old_of_new[cd.int_begin + l]] = -1;
        for (int32_t j = 0; j < cd.n_sh; ++j) loc_of_vtx[shl[j]] = -1;
        m.max_patch = std::max(m.max_patch, np);
        m.max_elem = std::max(m.max_elem, n_el);
        m.max_loc = std::max(m.max_loc, cd.n_loc);
        m.max_sh = std::max(m.max_sh, cd.n_sh);
        m.max_inc = std::max(m.max_inc, n_inc);
    }
    m.patch_total = patch_off;
    m.inc_total = inc_off;
    m.sh_total = sh_off;
    m.loc_total = node_off;
    m.incp_total = incp_off;

    // ---- partial slots of every shared node, in chunk order
    for (int64_t s = 0; s < m.n_shared; ++s) shr_cnt[s + 1] += shr_cnt[s];
    m.shr_ptr.assign(shr_cnt.begin(), shr_cnt.end());
    m.shr_slot.assign(m.shr_ptr.back(), 0);
    {
        std::vector<int32_t> fill(m.shr_ptr.begin(), m.shr_ptr.end() - 1);
        for (int c = 0; c < nc; ++c) {
            const ChunkDesc &cd = m.chunks[c];
            for (int32_t j = 0; j < cd.n_sh; ++j) {
                int64_t s = m.sh_ids[cd.sh_off + j] - m.n_int;
                m.shr_slot[fill[s]++] = cd.sh_off + j;
            }
        }
    }
    // partial sums are stored shared-node-major: chunk slot -> its position
    m.sh_dest.assign(m.sh_total, -1);
    for (size_t k = 0; k < m.shr_slot.size(); ++k) m.sh_dest[m.shr_slot[k]] = (int32_t)k;
    // the first chunk holding a shared node owns it: that chunk alone stores
    // the node's values in passes where every holder evaluates them
    m.sh_info.assign(m.sh_total * 4, 0);
    for (int64_t k = 0; k < m.sh_total; ++k) {
        const int32_t g = m.sh_ids[k];
        m.sh_info[4 * k] = g;
        if (g < 0) continue;
        const int64_t s = g - m.n_int;
        m.sh_info[4 * k + 1] = m.shr_ptr[s];
        m.sh_info[4 * k + 2] = m.shr_ptr[s + 1];
        m.sh_info[4 * k + 3] = m.shr_slot[m.shr_ptr[s]] == k ? 1 : 0;
    }
    if (dim == 3) return build_units(m);
    return "";
}

std::string build_units(PrepMesh &m) {
    if (m.dim != 3) return "paired-patch layout: 3D only";
    m.chunks_u.assign(m.n_chunks, ChunkUnits{});
    m.urec.clear();
    m.uelem.clear();
    m.unit_total = 0;
    m.max_unit = 0;
    struct Ref { int p, m; };
    std::vector<Ref> ps;
    std::vector<int> star;
    for (int c = 0; c < m.n_chunks; ++c) {
        const ChunkDesc &cd = m.chunks[c];
        ChunkUnits &cu = m.chunks_u[c];
        // patches by size, largest first (stable), paired two by two
        ps.clear();
        for (int q = 0; q < cd.n_patch; ++q) ps.push_back({q, (int)m.pids[(size_t)(cd.patch_off + q) * kPatchIds]});
        std::stable_sort(ps.begin(), ps.end(), [](const Ref &x, const Ref &y) { return x.m > y.m; });
        std::vector<std::array<int, 2>> units;
        for (size_t i = 0; i < ps.size();) {
            if (i + 1 < ps.size() && ps[i + 1].m == ps[i].m) {
                units.push_back({ps[i].p, ps[i + 1].p});
                i += 2;
            } else {
                units.push_back({ps[i].p, -1});   // paired with itself
                i += 1;
            }
        }
        // an even count per chunk: every chunk's records start and end on a
        // 16-byte boundary (bulk copies); the pad unit has no element (m = 0)
        if (units.size() & 1) units.push_back({-1, -1});
        const int nu = (int)units.size();
        cu.unit_off = (int32_t)m.unit_total;
        cu.n_unit = nu;
        star.assign(cd.n_loc, 0);
        for (int u = 0; u < nu; ++u) {
            uint32_t w[kURecWords] = {0};
            int32_t el[kPatchMax * 2];
            for (int k = 0; k < kPatchMax * 2; ++k) el[k] = -1;
            int pm = 0;
            for (int h = 0; h < 2 && units[u][0] >= 0; ++h) {
                const bool dup = units[u][h] < 0;
                const int q = dup ? units[u][0] : units[u][h];
                const uint16_t *rec = &m.pids[(size_t)(cd.patch_off + q) * kPatchIds];
                pm = rec[0];
                const int shift = 16 * h;
                w[0] = (uint32_t)pm | (dup ? kUnitDup : 0u);
                w[1] |= (uint32_t)rec[1] << shift;
                w[2] |= (uint32_t)rec[2] << shift;
                for (int j = 0; j <= pm; ++j) w[3 + j] |= (uint32_t)rec[3 + j] << shift;
                if (dup) continue;   // no element behind the duplicate half
                for (int j = 0; j < pm; ++j) {
                    el[2 * j + h] = m.elem_src[(size_t)(cd.patch_off + q) * kPatchMax + j];
                    // elements around each of the element's vertices (a, b, r_j, r_{j+1})
                    star[rec[1]]++;
                    star[rec[2]]++;
                    star[rec[3 + j]]++;
                    star[rec[4 + j]]++;
                }
            }
            for (int k = 0; k < kURecWords; ++k) m.urec.push_back(w[k]);
            for (int k = 0; k < kPatchMax * 2; ++k) m.uelem.push_back(el[k]);
        }
        int ms = 1;
        for (int l = 0; l < cd.n_loc; ++l) ms = std::max(ms, star[l]);
        cu.max_star = ms;
        m.unit_total += nu;
        m.max_unit = std::max(m.max_unit, nu);
    }
    return "";
}

std::string validate_prep(const PrepMesh &m, const int32_t *conn) {
    const int nv = m.nv;
    std::vector<int> seen_elem(m.n_elems, 0);
    std::vector<int32_t> owner(m.n_dofs, -1);
    for (int c = 0; c < m.n_chunks; ++c) {
        const ChunkDesc &cd = m.chunks[c];
        if (cd.patch_off % kPatchPad || cd.sh_off % kShPad || cd.incp_off % kIncpPad || cd.inc_off % kIncPad)
            return "segment not aligned";
        for (int32_t l = 0; l < cd.n_loc; ++l) {
            const int32_t want_g = l < cd.n_int ? cd.int_begin + l : m.sh_ids[cd.sh_off + l - cd.n_int];
            if (m.loc_node[cd.node_off + l] != want_g) return "local node maps to the wrong unknown";
            if (m.new_of_old[m.loc_orig[cd.node_off + l]] != want_g) return "local vertex maps to the wrong unknown";
        }
        std::vector<int> hits((size_t)cd.n_patch * kPatchSlots, 0);
        std::vector<int> slot_node((size_t)cd.n_patch * kPatchSlots, -1);
        int n_el = 0;
        for (int q = 0; q < cd.n_patch; ++q) {
            const uint16_t *rec = &m.pids[(int64_t)(cd.patch_off + q) * kPatchIds];
            const int pm = rec[0];
            if (pm < 1 || pm > kPatchMax) return "bad patch size";
            slot_node[q * kPatchSlots + 0] = rec[1];
            if (m.dim == 3) slot_node[q * kPatchSlots + 1] = rec[2];
            for (int j = 0; j <= pm; ++j) slot_node[q * kPatchSlots + 2 + j] = rec[3 + j];
            for (int j = 0; j < pm; ++j) {
                int32_t src = m.elem_src[(int64_t)(cd.patch_off + q) * kPatchMax + j];
                if (src < 0 || src >= m.n_elems) return "bad element source";
                seen_elem[src]++;
                ++n_el;
                std::vector<int32_t> want, have;
                for (int a = 0; a < nv; ++a) want.push_back(conn[(int64_t)src * nv + a]);
                have.push_back(m.loc_orig[cd.node_off + rec[1]]);
                if (m.dim == 3) have.push_back(m.loc_orig[cd.node_off + rec[2]]);
                have.push_back(m.loc_orig[cd.node_off + rec[3 + j]]);
                have.push_back(m.loc_orig[cd.node_off + rec[3 + j + 1]]);
                std::sort(want.begin(), want.end());
                std::sort(have.begin(), have.end());
                if (want != have) return "patch element does not match the mesh";
                for (int a = 0; a < nv; ++a) {
                    int32_t g = m.new_of_old[want[a]];
                    if (g < m.n_int) {
                        if (owner[g] != -1 && owner[g] != c) return "interior node in two chunks";
                        owner[g] = c;
                    }
                }
            }
            for (int j = pm; j < kPatchMax; ++j)
                if (m.elem_src[(int64_t)(cd.patch_off + q) * kPatchMax + j] != -1) return "stray element slot";
        }
        if (n_el != cd.n_elem) return "chunk element count mismatch";
        for (int32_t l = 0; l < cd.n_loc; ++l) {
            int b = m.incp[cd.incp_off + l], e = m.incp[cd.incp_off + l + 1];
            for (int k = b; k < e; ++k) {
                int idx = m.inc[cd.inc_off + k];
                if (idx >= cd.n_patch * kPatchSlots) return "bad incidence entry";
                if (slot_node[idx] != l) return "incidence/slot mismatch";
                hits[idx]++;
            }
        }
        for (size_t k = 0; k < hits.size(); ++k)
            if ((slot_node[k] >= 0) != (hits[k] == 1)) return "slot not covered exactly once";
    }
    for (int64_t e = 0; e < m.n_elems; ++e)
        if (seen_elem[e] != 1) return "element not placed exactly once";
    std::vector<int> slot_hits(m.sh_total, 0);
    for (int64_t s = 0; s < m.n_shared; ++s)
        for (int32_t k = m.shr_ptr[s]; k < m.shr_ptr[s + 1]; ++k) {
            int32_t slot = m.shr_slot[k];
            if (m.sh_ids[slot] != m.n_int + s) return "partial slot maps to wrong node";
            if (m.sh_dest[slot] != k) return "partial destination is not the inverse slot map";
            slot_hits[slot]++;
        }
    for (int64_t k = 0; k < m.sh_total; ++k)
        if ((m.sh_ids[k] >= 0) != (slot_hits[k] == 1)) return "partial slots not a bijection";
    if ((int64_t)m.sh_info.size() != 4 * m.sh_total) return "slot info missing";
    std::vector<int> owners(m.n_shared, 0);
    for (int64_t k = 0; k < m.sh_total; ++k) {
        const int32_t *si = &m.sh_info[4 * k];
        if (si[0] != m.sh_ids[k]) return "slot info node mismatch";
        if (si[0] < 0) {
            if (si[1] || si[2] || si[3]) return "slot info on a pad slot";
            continue;
        }
        const int64_t s = si[0] - m.n_int;
        if (si[1] != m.shr_ptr[s] || si[2] != m.shr_ptr[s + 1]) return "slot info range mismatch";
        if (si[3]) owners[s]++;
    }
    for (int64_t s = 0; s < m.n_shared; ++s)
        if (owners[s] != 1) return "shared node without exactly one owner";
    return "";
}

}  // namespace ps
