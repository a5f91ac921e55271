// Device data layout of one preprocessed mesh, shared by the host
// preprocessing (mesh_prep.cpp) and the CUDA kernels.
//
// Elements are partitioned into "chunks" of consecutive elements along a Morton
// curve of their centroids, and inside a chunk into star-shaped patches.  Nodes touched by exactly one chunk are that
// chunk's interior nodes; they are numbered contiguously per chunk, so the
// chunk owns their rows outright.  Nodes touched by several chunks ("shared")
// are numbered after all interior nodes.  A chunk computes its element
// contributions in shared memory, sums them per local node through a fixed
// incidence list (deterministic, no atomics), writes its interior rows
// directly and writes one partial sum per shared local node, into a
// shared-node-major array (the partials of one shared node are contiguous); a
// second pass adds the partial sums of every shared node in chunk order.
//
// Every per-chunk segment starts on a 16-byte boundary so that it can be moved
// into shared memory with one cp.async.bulk copy.
#pragma once
#include <stdint.h>

namespace ps {

constexpr int kPatchMax = 6;     // elements per patch (star) at most
constexpr int kPatchIds = 12;    // u16 per patch record: m, a, b, ring[0..m], padding
constexpr int kPatchSlots = 9;   // contribution slots per patch: a, b, ring[0..6]
// FP64 element geometry per patch slot: 3D G_AB, G_A0, G_A1, G_B0, G_B1, G_01, |det|, pad;
// 2D G_A0, G_A1, G_01, |det| (G_ab = c_a.c_b / (d! |det|), c_a the cofactor vectors)
template <int D>
constexpr int kGeoWords = D == 3 ? 8 : 4;
constexpr int kPatchPad = 4;     // patch segments padded to 4 patches (96 B)
constexpr int kIncPad = 8;       // incidence segments padded to 8 u16
constexpr int kIncpPad = 8;      // incidence-pointer segments padded to 8 u16
constexpr int kShPad = 4;        // shared-id segments padded to 4 int32
constexpr int kMaxChunkPatches = 65535 / kPatchSlots;  // slot ids fit in u16
constexpr int kChunkThreads = 256;  // threads of a block that processes a chunk

// Elements of a chunk are grouped into "patches": the elements around one
// pivot (an edge (a, b) in 3D, a vertex a in 2D), ordered so that element j of
// the patch is (a, b, ring[j], ring[j+1]) in 3D and (a, ring[j], ring[j+1]) in
// 2D, j = 0..m-1.  A closed star repeats ring[0] as ring[m].  An element that
// joins no star is a patch of one (m = 1).  Patch record (u16): [0] = m,
// [1] = a, [2] = b (3D), [3 + j] = ring[j], j = 0..m; all local node ids.
// Contribution slots: 0 -> a, 1 -> b, 2 + j -> ring[j].

// Paired-patch layout of the FP32 3D CG operator kernel (k_cg2_units): the
// star patches of a chunk are taken two at a time ("units"), two patches of
// the same size m, so that one thread evaluates both with packed FP32x2
// arithmetic (one half per patch).  Units are ordered by m, largest first; a
// size class with an odd count pairs its last patch with itself, and that
// unit's second half is flagged so its contributions are dropped.  Each
// chunk holds an even number of units (a pad unit with m = 0 and no element
// makes it even), so that a chunk's unit records (40 bytes each) and
// beta*dt^2/6 values (48 bytes each) start and end on 16-byte boundaries.
//   unit record (u32): [0] = m | kUnitDup (second half duplicate),
//                      [1] = (a | a' << 16), [2] = (b | b' << 16),
//                      [3 + j] = (r_j | r'_j << 16), j = 0..m; local node ids
// Node sums are fixed-point shared-memory integer atomics (exact additions:
// the result does not depend on their order), so no incidence list is needed.
constexpr int kURecWords = 10;
constexpr uint32_t kUnitDup = 0x100u;
struct ChunkUnits {
    int32_t unit_off;   // first unit of the chunk
    int32_t n_unit;
    int32_t max_star;   // most elements of the chunk around one of its nodes
    int32_t pad;
};
static_assert(sizeof(ChunkUnits) == 16, "ChunkUnits layout");

struct ChunkDesc {
    int32_t patch_off;  // first (padded) patch of the chunk
    int32_t n_patch;
    int32_t node_off;   // first entry of the chunk's node block
    int32_t n_loc;      // local nodes = n_int + n_sh
    int32_t n_int;      // interior nodes: local 0..n_int-1 = new ids int_begin + l
    int32_t int_begin;
    int32_t sh_off;     // first entry in sh_ids / partial slots (padded)
    int32_t n_sh;       // shared local nodes: local n_int + j -> sh_ids[sh_off + j]
    int32_t incp_off;   // first entry of the chunk's incidence pointers (padded)
    int32_t inc_off;    // first entry of the chunk's incidence list (padded)
    int32_t n_inc;      // incidence entries (patch * kPatchSlots + slot)
    int32_t n_elem;
};
static_assert(sizeof(ChunkDesc) == 48, "ChunkDesc layout");

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

}  // namespace ps
