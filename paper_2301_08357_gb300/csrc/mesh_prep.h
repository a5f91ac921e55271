// Host preprocessing of a primal simplex mesh (Section 3.1) into the chunked
// device layout described in layout.h.
#pragma once
#include <stdint.h>

#include <string>
#include <vector>

#include "layout.h"

namespace ps {

struct PrepOptions {
    int chunk_elems = 0;      // 0 = auto
    int chunk_nodes_max = 0;  // 0 = auto
    // periodic boundaries by vertex merging (Section 3.6): master[i] is the
    // vertex whose unknown vertex i shares (master[master[i]] == master[i]);
    // nullptr = no merging
    const int32_t *periodic = nullptr;
    // split each of the first `split_lead` chunks into two halves (Morton
    // order), when the mesh has at least four times as many chunks: the
    // blocks of the first wave then end at different times, so the blocks
    // resident on an SM do not stay in step (0 = no split)
    int split_lead = 0;
};

struct PrepMesh {
    int dim = 0, nv = 0;
    int64_t n_nodes = 0, n_elems = 0, n_free = 0;
    int64_t n_dofs = 0;       // unknowns: n_nodes minus merged periodic vertices
    int n_chunks = 0;
    int64_t n_int = 0;        // interior nodes (new ids 0..n_int-1)
    int64_t n_shared = 0;     // shared nodes (new ids n_int..n_nodes-1)
    int64_t patch_total = 0;  // padded patch records
    int64_t n_patches = 0;    // real patches
    int64_t inc_total = 0;    // padded incidence entries
    int64_t loc_total = 0;    // sum of n_loc
    int64_t incp_total = 0;
    int64_t sh_total = 0;     // padded shared-id slots (= partial slots)
    int max_patch = 0, max_loc = 0, max_sh = 0, max_inc = 0, max_elem = 0;

    std::vector<int32_t> new_of_old;               // [n_nodes] unknown of each vertex
    std::vector<int32_t> old_of_new;               // [n_dofs] master vertex of each unknown
    std::vector<uint8_t> dirichlet_new;            // [n_dofs]
    std::vector<int32_t> slave_ptr, slave;         // [n_dofs + 1], merged vertices per unknown (empty: no merging)
    std::vector<ChunkDesc> chunks;                 // [n_chunks]
    std::vector<uint16_t> pids;                    // [patch_total * kPatchIds]
    std::vector<int32_t> elem_src;                 // [patch_total * kPatchMax] original element, -1 unused
    std::vector<uint16_t> incp;                    // [incp_total]
    std::vector<uint16_t> inc;                     // [inc_total] patch * kPatchSlots + slot
    std::vector<int32_t> sh_ids;                   // [sh_total], -1 pad
    std::vector<int32_t> loc_node;                 // [loc_total] unknown (new id) of each local node
    std::vector<int32_t> loc_orig;                 // [loc_total] vertex (caller's id) of each local node
    std::vector<double> loc_rel;                   // [loc_total * dim] coords - chunk origin
    std::vector<int32_t> shr_ptr;                  // [n_shared + 1]
    std::vector<int32_t> shr_slot;                 // chunk-major slot of each shared-node-major partial
    std::vector<int32_t> sh_dest;                  // [sh_total] shared-node-major position of a chunk slot, -1 pad
    // [sh_total * 4] per chunk slot: node id, begin and end of the node's
    // partial-sum range, 1 on the owner slot (the node's first chunk); pads -1, 0, 0, 0
    std::vector<int32_t> sh_info;

    // paired-patch layout (layout.h; 3D only, empty in 2D)
    std::vector<ChunkUnits> chunks_u;              // [n_chunks]
    std::vector<uint32_t> urec;                    // [unit_total * kURecWords]
    std::vector<int32_t> uelem;                    // [unit_total * kPatchMax * 2] element of (tet j, half h), -1 none
    int64_t unit_total = 0;
    int max_unit = 0;
};

// Build the paired-patch layout from a prepared 3D mesh (its patch records
// and element map).  Returns "" on success.
std::string build_units(PrepMesh &m);

// Returns "" on success, else an error message (bad input).
std::string prepare_mesh(int dim, int64_t n_nodes, const double *coords, int64_t n_elems,
                         const int32_t *conn, const uint8_t *dirichlet, const PrepOptions &opt,
                         PrepMesh &out);

// Checks the invariants the kernels rely on (used by the tests through the ABI
// debug hook): every element sits in exactly one patch slot with the patch's
// vertex pattern, every used contribution slot appears once in the incidence
// list of its node, interior nodes are touched by one chunk only, partial
// slots are a bijection.
std::string validate_prep(const PrepMesh &m, const int32_t *conn_original);

}  // namespace ps
