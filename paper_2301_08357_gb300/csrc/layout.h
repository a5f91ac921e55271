// Device data layout of one preprocessed mesh, shared by the host
// preprocessing (mesh_prep.cpp) and the CUDA kernels.
//
// Elements are partitioned into "chunks" of consecutive elements along a Morton
// curve of their centroids.  Nodes touched by exactly one chunk are that
// chunk's interior nodes; they are numbered contiguously per chunk, so the
// chunk owns their rows outright.  Nodes touched by several chunks ("shared")
// are numbered after all interior nodes.  A chunk computes its element
// contributions in shared memory, sums them per local node through a fixed
// incidence list (deterministic, no atomics), writes its interior rows
// directly and writes one partial sum per shared local node; a second pass
// adds the partial sums of every shared node in a fixed order.
//
// Every per-chunk segment starts on a 16-byte boundary so that it can be moved
// into shared memory with one cp.async.bulk copy.
#pragma once
#include <stdint.h>

namespace ps {

constexpr int kElemPad = 8;     // element segments padded to 8 elements
constexpr int kIncpPad = 8;     // incidence-pointer segments padded to 8 u16
constexpr int kShPad = 4;       // shared-id segments padded to 4 int32
constexpr int kMaxChunkElems = 16383;  // slot = 4 * e + v must fit in u16

struct ChunkDesc {
    int32_t elem_off;   // first (padded) element of the chunk
    int32_t n_elem;
    int32_t node_off;   // first entry of the chunk's node block
    int32_t n_loc;      // local nodes = n_int + n_sh
    int32_t n_int;      // interior nodes: local 0..n_int-1 = new ids int_begin + l
    int32_t int_begin;
    int32_t sh_off;     // first entry in sh_ids / partial slots (padded)
    int32_t n_sh;       // shared local nodes: local n_int + j -> sh_ids[sh_off + j]
    int32_t incp_off;   // first entry of the chunk's incidence pointers (padded)
    int32_t pad0, pad1, pad2;
};
static_assert(sizeof(ChunkDesc) == 48, "ChunkDesc layout");

inline int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

}  // namespace ps
