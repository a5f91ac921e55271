// Serving loop (filled in with the continuous-batching worker).
#include "../../include/pressure.h"

extern "C" int ps_server_create(ps_ctx *, const ps_server_opts *, ps_server **out) {
    if (out) *out = nullptr;
    return PS_ESTATE;
}
extern "C" void ps_server_destroy(ps_server *) {}
extern "C" int ps_server_add_case(ps_server *, ps_mesh *, const double *, int32_t *) { return PS_ESTATE; }
extern "C" int ps_solve_submit(ps_server *, int32_t, const double *, const double *, ps_ticket *) { return PS_ESTATE; }
extern "C" int ps_solve_poll(ps_server *, ps_ticket, ps_solve_info *, double *) { return PS_ESTATE; }
extern "C" int ps_solve_wait(ps_server *, ps_ticket, double, ps_solve_info *, double *) { return PS_ESTATE; }
extern "C" int ps_server_release(ps_server *, ps_ticket) { return PS_ESTATE; }
extern "C" int ps_server_get_stats(ps_server *, ps_server_stats *) { return PS_ESTATE; }
