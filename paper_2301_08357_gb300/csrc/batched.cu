// Batched persistent solver (placeholder until the persistent kernel lands).
#include "../../include/pressure.h"
#include "internal.h"
namespace ps {
int batched_set_attrs() { return 0; }
void batched_release_mesh(ps_mesh *) {}
}  // namespace ps

extern "C" int ps_batch_solve(ps_mesh *const *, int, const double *const *, double *const *,
                              const ps_solve_opts *, ps_solve_info *, void *) {
    return PS_ESTATE;
}
