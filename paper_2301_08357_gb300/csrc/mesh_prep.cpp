// Host preprocessing: Morton chunking, node renumbering, local connectivity.
// See layout.h for the layout this produces.
#include "mesh_prep.h"

#include <algorithm>
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

}  // namespace

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
    for (int64_t e = 0; e < n_elems; ++e) {
        double d = simplex_det(dim, coords, conn + e * nv);
        if (!(std::fabs(d) > vol_floor)) return "element of zero volume";
        for (int a = 0; a < nv; ++a)
            for (int b = a + 1; b < nv; ++b)
                if (conn[e * nv + a] == conn[e * nv + b]) return "repeated vertex in element";
    }

    // ---- Morton order of element centroids
    std::vector<uint64_t> key(n_elems);
    std::vector<int32_t> order(n_elems);
    const int bits = dim == 3 ? 21 : 31;
    const double scale = (double)((1ULL << bits) - 1) / ext;
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
        // aim for ~8 chunks per SM of a 152-SM part, 128..1024 elements each
        int64_t t = n_elems / 1216;
        t = std::max<int64_t>(128, std::min<int64_t>(1024, t));
        ec = (int)round_up(t, 32);
    }
    ec = std::max(1, std::min(ec, kMaxChunkElems));
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
    const int nc = (int)chunk_begin.size() - 1;
    m.n_chunks = nc;

    // ---- classify nodes: interior (one chunk) or shared
    std::vector<int32_t> last(n_nodes, -1);
    std::vector<uint8_t> shared(n_nodes, 0);
    for (int c = 0; c < nc; ++c)
        for (int64_t k = chunk_begin[c]; k < chunk_begin[c + 1]; ++k) {
            const int32_t *v = conn + (int64_t)order[k] * nv;
            for (int a = 0; a < nv; ++a) {
                if (last[v[a]] != c) {
                    if (last[v[a]] != -1) shared[v[a]] = 1;
                    last[v[a]] = c;
                }
            }
        }
    for (int64_t i = 0; i < n_nodes; ++i)
        if (last[i] == -1) return "node not used by any element";

    // ---- renumber: interior nodes per chunk, then shared nodes
    m.new_of_old.assign(n_nodes, -1);
    m.chunks.resize(nc);
    int32_t next = 0;
    for (int c = 0; c < nc; ++c) {
        ChunkDesc &cd = m.chunks[c];
        std::memset(&cd, 0, sizeof(cd));
        cd.int_begin = next;
        for (int64_t k = chunk_begin[c]; k < chunk_begin[c + 1]; ++k) {
            const int32_t *v = conn + (int64_t)order[k] * nv;
            for (int a = 0; a < nv; ++a)
                if (!shared[v[a]] && m.new_of_old[v[a]] < 0) m.new_of_old[v[a]] = next++;
        }
        cd.n_int = next - cd.int_begin;
    }
    m.n_int = next;
    for (int c = 0; c < nc; ++c)
        for (int64_t k = chunk_begin[c]; k < chunk_begin[c + 1]; ++k) {
            const int32_t *v = conn + (int64_t)order[k] * nv;
            for (int a = 0; a < nv; ++a)
                if (shared[v[a]] && m.new_of_old[v[a]] < 0) m.new_of_old[v[a]] = next++;
        }
    m.n_shared = next - m.n_int;
    m.old_of_new.assign(n_nodes, 0);
    m.dirichlet_new.assign(n_nodes, 0);
    for (int64_t i = 0; i < n_nodes; ++i) {
        m.old_of_new[m.new_of_old[i]] = (int32_t)i;
        m.dirichlet_new[m.new_of_old[i]] = dirichlet ? (dirichlet[i] != 0) : 0;
    }
    m.n_free = 0;
    for (int64_t i = 0; i < n_nodes; ++i) m.n_free += m.dirichlet_new[i] == 0;

    // ---- per-chunk local structure
    int64_t elem_off = 0, node_off = 0, sh_off = 0, incp_off = 0;
    for (int c = 0; c < nc; ++c) {
        ChunkDesc &cd = m.chunks[c];
        cd.n_elem = (int32_t)(chunk_begin[c + 1] - chunk_begin[c]);
        cd.elem_off = (int32_t)elem_off;
        elem_off += round_up(cd.n_elem, kElemPad);
    }
    m.elem_total = elem_off;
    m.elem_src.assign(m.elem_total, -1);
    m.lconn.assign(m.elem_total * 4, 0);
    m.inc.assign(m.elem_total * 4, 0);
    std::vector<int32_t> loc_of_new(n_nodes, -1);
    std::vector<int32_t> shl;
    std::vector<std::vector<int32_t>> node_slots;   // unused placeholder to keep code plain
    std::vector<int32_t> shr_cnt(m.n_shared + 1, 0);
    for (int c = 0; c < nc; ++c) {
        ChunkDesc &cd = m.chunks[c];
        // shared local nodes, ascending new id
        shl.clear();
        for (int64_t k = chunk_begin[c]; k < chunk_begin[c + 1]; ++k) {
            const int32_t *v = conn + (int64_t)order[k] * nv;
            for (int a = 0; a < nv; ++a) {
                int32_t g = m.new_of_old[v[a]];
                if (g >= m.n_int && loc_of_new[g] != -2) { loc_of_new[g] = -2; shl.push_back(g); }
            }
        }
        std::sort(shl.begin(), shl.end());
        cd.n_sh = (int32_t)shl.size();
        cd.n_loc = cd.n_int + cd.n_sh;
        cd.node_off = (int32_t)node_off;
        cd.sh_off = (int32_t)sh_off;
        cd.incp_off = (int32_t)incp_off;
        for (int32_t l = 0; l < cd.n_int; ++l) loc_of_new[cd.int_begin + l] = l;
        for (int32_t j = 0; j < cd.n_sh; ++j) {
            loc_of_new[shl[j]] = cd.n_int + j;
            m.sh_ids.push_back(shl[j]);
            shr_cnt[shl[j] - m.n_int + 1]++;
        }
        for (int64_t j = cd.n_sh; j < round_up(cd.n_sh, kShPad); ++j) m.sh_ids.push_back(-1);
        sh_off += round_up(cd.n_sh, kShPad);
        node_off += cd.n_loc;
        // local connectivity
        for (int32_t e = 0; e < cd.n_elem; ++e) {
            int32_t src = order[chunk_begin[c] + e];
            m.elem_src[cd.elem_off + e] = src;
            for (int a = 0; a < nv; ++a) {
                int32_t l = loc_of_new[m.new_of_old[conn[(int64_t)src * nv + a]]];
                m.lconn[(int64_t)(cd.elem_off + e) * 4 + a] = (uint16_t)l;
            }
        }
        // incidence lists: counting sort of slots 4e+a by local node
        std::vector<int32_t> cnt(cd.n_loc + 1, 0);
        for (int32_t e = 0; e < cd.n_elem; ++e)
            for (int a = 0; a < nv; ++a) cnt[m.lconn[(int64_t)(cd.elem_off + e) * 4 + a] + 1]++;
        for (int32_t l = 0; l < cd.n_loc; ++l) cnt[l + 1] += cnt[l];
        for (int32_t l = 0; l <= cd.n_loc; ++l) m.incp.push_back((uint16_t)cnt[l]);
        for (int64_t j = cd.n_loc + 1; j < round_up(cd.n_loc + 1, kIncpPad); ++j)
            m.incp.push_back((uint16_t)cnt[cd.n_loc]);
        incp_off += round_up(cd.n_loc + 1, kIncpPad);
        std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
        for (int32_t e = 0; e < cd.n_elem; ++e)
            for (int a = 0; a < nv; ++a) {
                int l = m.lconn[(int64_t)(cd.elem_off + e) * 4 + a];
                m.inc[(int64_t)cd.elem_off * 4 + fill[l]++] = (uint16_t)(4 * e + a);
            }
        // node block bookkeeping (coordinates relative to the chunk origin)
        int32_t origin_new = cd.n_loc > 0 ? (cd.n_int > 0 ? cd.int_begin : shl[0]) : 0;
        const double *o = coords + (int64_t)m.old_of_new[origin_new] * dim;
        for (int32_t l = 0; l < cd.n_loc; ++l) {
            int32_t g = l < cd.n_int ? cd.int_begin + l : shl[l - cd.n_int];
            m.loc_node.push_back(g);
            m.loc_chunk.push_back(c);
            const double *p = coords + (int64_t)m.old_of_new[g] * dim;
            for (int k = 0; k < dim; ++k) m.loc_rel.push_back(p[k] - o[k]);
        }
        for (int32_t l = 0; l < cd.n_int; ++l) loc_of_new[cd.int_begin + l] = -1;
        for (int32_t j = 0; j < cd.n_sh; ++j) loc_of_new[shl[j]] = -1;
        m.max_elem = std::max(m.max_elem, cd.n_elem);
        m.max_loc = std::max(m.max_loc, cd.n_loc);
        m.max_sh = std::max(m.max_sh, cd.n_sh);
    }
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
    return "";
}

std::string validate_prep(const PrepMesh &m, const int32_t *conn) {
    const int nv = m.nv;
    std::vector<int> seen_elem(m.n_elems, 0);
    std::vector<int32_t> owner(m.n_nodes, -1);
    for (int c = 0; c < m.n_chunks; ++c) {
        const ChunkDesc &cd = m.chunks[c];
        if (cd.elem_off % kElemPad || cd.sh_off % kShPad || cd.incp_off % kIncpPad)
            return "segment not aligned";
        std::vector<int> hits((size_t)cd.n_elem * 4, 0);
        for (int32_t l = 0; l < cd.n_loc; ++l) {
            int b = m.incp[cd.incp_off + l], e = m.incp[cd.incp_off + l + 1];
            for (int k = b; k < e; ++k) {
                int slot = m.inc[(int64_t)cd.elem_off * 4 + k];
                int el = slot / 4, a = slot % 4;
                if (el >= cd.n_elem || a >= nv) return "bad slot";
                if (m.lconn[(int64_t)(cd.elem_off + el) * 4 + a] != l) return "slot/local mismatch";
                hits[slot]++;
            }
        }
        for (int32_t e = 0; e < cd.n_elem; ++e) {
            for (int a = 0; a < nv; ++a)
                if (hits[4 * e + a] != 1) return "slot not covered once";
            int32_t src = m.elem_src[cd.elem_off + e];
            if (src < 0 || src >= m.n_elems) return "bad element source";
            seen_elem[src]++;
            for (int a = 0; a < nv; ++a) {
                int l = m.lconn[(int64_t)(cd.elem_off + e) * 4 + a];
                int32_t g = l < cd.n_int ? cd.int_begin + l : m.sh_ids[cd.sh_off + l - cd.n_int];
                if (m.old_of_new[g] != conn[(int64_t)src * nv + a]) return "connectivity mismatch";
                if (g < m.n_int) {
                    if (owner[g] != -1 && owner[g] != c) return "interior node in two chunks";
                    owner[g] = c;
                }
            }
        }
    }
    for (int64_t e = 0; e < m.n_elems; ++e)
        if (seen_elem[e] != 1) return "element not placed exactly once";
    std::vector<int> slot_hits(m.sh_total, 0);
    for (int64_t s = 0; s < m.n_shared; ++s)
        for (int32_t k = m.shr_ptr[s]; k < m.shr_ptr[s + 1]; ++k) {
            int32_t slot = m.shr_slot[k];
            if (m.sh_ids[slot] != m.n_int + s) return "partial slot maps to wrong node";
            slot_hits[slot]++;
        }
    for (int64_t k = 0; k < m.sh_total; ++k)
        if ((m.sh_ids[k] >= 0) != (slot_hits[k] == 1)) return "partial slots not a bijection";
    return "";
}

}  // namespace ps
