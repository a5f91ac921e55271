// Serving loop: continuous batching of pressure-solve requests from many
// simulated cases (see include/pressure.h, "serving").
//
// One worker thread owns a CUDA stream and a batch plan.  Between epochs it
// admits queued requests (one in flight per case, at most max_slots in flight,
// the sum of in-flight workspace bytes within the HBM budget), stages their
// inputs on its stream (right-hand side; a drifted beta with the element
// coefficients and the Jacobi diagonal updated on the device), solves the
// admitted requests of cases at or above the size threshold (single_nodes)
// alone to convergence with the single-solve engine, rebuilds the plan when
// the set of batched in-flight requests changed (a request already in flight
// keeps its device state; the plan keeps its buffers), runs one epoch of the
// batched engine for every batched in-flight request, and completes the
// requests whose solve finished.  A request warm-starts from the pressure its
// case left on the device.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/pressure.h"
#include "batched.h"

using namespace ps;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Req {
    ps_ticket id = 0;
    int32_t case_id = 0;
    std::vector<double> b, beta, x;
    int status = PS_PENDING;
    ps_solve_info info;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

struct Case {
    ps_mesh *mesh = nullptr;
    std::vector<DevAlloc> allocs;
    double *b_dev = nullptr, *x_dev = nullptr;
    double *beta_dev = nullptr;      // a request's drifted beta, staged for the on-device update
    bool single = false;             // requests run alone in the single-solve engine (single_nodes)
    std::deque<Req *> queue;
    Req *running = nullptr;
    int64_t ws_bytes = 0;
};

}  // namespace

struct ps_server {
    ps_ctx *ctx = nullptr;
    ps_server_opts opts;
    std::thread worker;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    cudaStream_t stream = nullptr;
    std::vector<Case> cases;
    std::map<ps_ticket, Req *> reqs;
    ps_ticket next_ticket = 1;
    ps_server_stats st;
    int64_t in_flight_bytes = 0;
    // worker-only
    BatchPlan plan;
    std::vector<int> plan_cases;
};

static int64_t server_budget(const ps_server *s) {
    if (s->opts.hbm_budget_bytes) return (int64_t)s->opts.hbm_budget_bytes;
    return 0;  // no cap on in-flight workspaces
}

static void finish_req(ps_server *s, Case &c, Req *r, int status, const ps_solve_info *info) {
    r->status = status;
    if (info) r->info = *info;
    r->t_done = now_s();
    r->info.seconds = r->t_done - r->t_submit;
    r->info.queue_seconds = r->t_admit > 0 ? r->t_admit - r->t_submit : r->info.seconds;
    if (status == PS_OK)
        s->st.completed++;
    else
        s->st.failed++;
    c.running = nullptr;
}

static void worker_main(ps_server *s) {
    cudaSetDevice(s->ctx->device);
    std::vector<int> admitted;
    for (;;) {
        admitted.clear();
        bool membership_changed = false;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            for (;;) {
                if (s->stop) break;
                // admission: oldest queued request first, one per case
                const int64_t budget = server_budget(s);
                for (;;) {
                    int best = -1;
                    for (size_t ci = 0; ci < s->cases.size(); ++ci) {
                        Case &c = s->cases[ci];
                        if (c.running || c.queue.empty()) continue;
                        if (best < 0 || c.queue.front()->t_submit < s->cases[best].queue.front()->t_submit)
                            best = (int)ci;
                    }
                    if (best < 0) break;
                    Case &c = s->cases[best];
                    if (s->st.in_flight >= s->opts.max_slots) break;
                    if (budget && s->in_flight_bytes + c.ws_bytes > budget) {
                        if (s->st.in_flight == 0) {   // can never fit: fail it
                            Req *r = c.queue.front();
                            c.queue.pop_front();
                            s->st.queued--;
                            c.running = r;
                            finish_req(s, c, r, PS_ENOMEM, nullptr);
                            s->cv_done.notify_all();
                            continue;
                        }
                        break;
                    }
                    Req *r = c.queue.front();
                    c.queue.pop_front();
                    s->st.queued--;
                    c.running = r;
                    r->t_admit = now_s();
                    s->st.in_flight++;
                    s->st.peak_in_flight = std::max(s->st.peak_in_flight, s->st.in_flight);
                    s->in_flight_bytes += c.ws_bytes;
                    admitted.push_back(best);
                }
                if (s->st.in_flight > 0) break;
                s->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            }
            if (s->stop) break;
        }
        const double t0 = now_s();
        std::lock_guard<std::mutex> ctx_lk(s->ctx->mu);
        int rc = PS_OK;
        // stage the admitted requests' inputs, in stream order on the
        // worker's stream (no allocation, no device-wide synchronisation)
        for (int ci : admitted) {
            Case &c = s->cases[ci];
            Req *r = c.running;
            if (!r->beta.empty()) {
                // the enthalpy drifted: new beta (same alpha, dt^2), then the
                // element coefficients and the Jacobi diagonal on the device
                // (the same kernels as ps_coeff_set_beta)
                if (cudaMemcpyAsync(c.beta_dev, r->beta.data(), r->beta.size() * 8, cudaMemcpyHostToDevice,
                                    s->stream) != cudaSuccess)
                    rc = PS_ECUDA;
                else
                    rc = beta_update_device(c.mesh, c.beta_dev, c.mesh->dt2, s->stream, true);
            }
            if (rc == PS_OK &&
                cudaMemcpyAsync(c.b_dev, r->b.data(), r->b.size() * 8, cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
                rc = PS_ECUDA;
            membership_changed = true;
        }
        // requests of large meshes: each solved alone, to convergence, by the
        // single-solve engine on the worker's stream, warm-starting from the
        // case's resident pressure (no epochs shared with the batch)
        std::vector<std::pair<int, ps_solve_info>> done;
        for (int ci : admitted) {
            Case &c = s->cases[ci];
            if (!c.single || rc != PS_OK) continue;
            ps_solve_info inf;
            const int sr = pressure_solve_locked(c.mesh, c.b_dev, c.x_dev, &s->opts.opts, &inf, s->stream);
            if (sr != PS_OK && sr != PS_ENOTCONV && sr != PS_EBREAKDOWN) {
                rc = sr;
                break;
            }
            inf.status = sr;
            c.running->x.resize(c.running->b.size());
            if (cudaMemcpyAsync(c.running->x.data(), c.x_dev, c.running->x.size() * 8, cudaMemcpyDeviceToHost,
                                s->stream) != cudaSuccess ||
                cudaStreamSynchronize(s->stream) != cudaSuccess) {
                rc = PS_ECUDA;
                break;
            }
            done.push_back({ci, inf});
            std::lock_guard<std::mutex> lk(s->mu);
            s->st.single_solves++;
        }
        const size_t n_single_done = done.size();   // complete, results on the host
        // (re)build the plan over the in-flight batched requests, keeping the
        // device state of requests already running
        if (rc == PS_OK) {
            std::vector<int> cur;
            {
                std::lock_guard<std::mutex> lk(s->mu);
                for (size_t ci = 0; ci < s->cases.size(); ++ci)
                    if (s->cases[ci].running && !s->cases[ci].single) cur.push_back((int)ci);
            }
            if (cur != s->plan_cases) membership_changed = true;
            if (membership_changed) {
                std::vector<BState> keep(cur.size());
                std::vector<char> have(cur.size(), 0);
                for (size_t k = 0; k < cur.size(); ++k)
                    for (size_t j = 0; j < s->plan_cases.size(); ++j)
                        if (s->plan_cases[j] == cur[k] &&
                            std::find(admitted.begin(), admitted.end(), cur[k]) == admitted.end()) {
                            keep[k] = s->plan.h_st[j];
                            have[k] = 1;
                        }
                std::vector<ps_mesh *> ms;
                for (int ci : cur) ms.push_back(s->cases[ci].mesh);
                s->plan_cases = cur;
                if (cur.empty()) {
                    batch_plan_free(s->plan);
                } else {
                    rc = batch_plan_build(s->ctx, ms.data(), (int)ms.size(), s->opts.epoch_iters, s->opts.opts,
                                          s->stream, s->plan);
                    for (size_t k = 0; k < cur.size() && rc == PS_OK; ++k) {
                        Case &c = s->cases[cur[k]];
                        batch_arm(s->plan, (int)k, c.b_dev, c.x_dev, s->opts.opts);
                        if (have[k]) s->plan.h_st[k] = keep[k];
                    }
                    if (rc == PS_OK) rc = batch_upload_states(s->plan, s->stream);
                }
            }
        }
        if (rc == PS_OK && !s->plan_cases.empty()) rc = batch_epoch(s->plan, s->stream);
        // completions of the batched requests
        if (rc == PS_OK) {
            for (size_t k = 0; k < s->plan_cases.size(); ++k) {
                if (s->plan.h_st[k].phase != kPhDone) continue;
                Case &c = s->cases[s->plan_cases[k]];
                if (!c.running) continue;
                ps_solve_info inf;
                batch_info(s->plan, (int)k, &inf);
                c.running->x.resize(c.running->b.size());
                if (cudaMemcpyAsync(c.running->x.data(), c.x_dev, c.running->x.size() * 8, cudaMemcpyDeviceToHost,
                                    s->stream) != cudaSuccess)
                    rc = PS_ECUDA;
                done.push_back({s->plan_cases[k], inf});
            }
            if (!done.empty() && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = PS_ECUDA;
        }
        std::lock_guard<std::mutex> lk(s->mu);
        s->st.epochs++;
        s->st.busy_seconds += now_s() - t0;
        if (rc != PS_OK) {
            // the single-lane requests solved before the failure keep their
            // results; every other in-flight request fails; keep serving the
            // queue
            for (size_t k = 0; k < n_single_done; ++k) {
                Case &c = s->cases[done[k].first];
                s->in_flight_bytes -= c.ws_bytes;
                s->st.in_flight--;
                finish_req(s, c, c.running, done[k].second.status, &done[k].second);
            }
            for (size_t ci = 0; ci < s->cases.size(); ++ci) {
                Case &c = s->cases[ci];
                if (!c.running) continue;
                s->in_flight_bytes -= c.ws_bytes;
                s->st.in_flight--;
                finish_req(s, c, c.running, rc, nullptr);
            }
            batch_plan_free(s->plan);
            s->plan_cases.clear();
        } else {
            for (auto &d : done) {
                Case &c = s->cases[d.first];
                s->in_flight_bytes -= c.ws_bytes;
                s->st.in_flight--;
                finish_req(s, c, c.running, d.second.status, &d.second);
            }
        }
        if (!done.empty() || rc != PS_OK) s->cv_done.notify_all();
    }
}

extern "C" int ps_server_create(ps_ctx *ctx, const ps_server_opts *opts, ps_server **out) {
    if (!ctx || !out) return PS_EINVAL;
    *out = nullptr;
    ps_server *s = new (std::nothrow) ps_server();
    if (!s) return PS_ENOMEM;
    s->ctx = ctx;
    if (opts) s->opts = *opts; else std::memset(&s->opts, 0, sizeof(s->opts));
    if (!opts) ps_solve_opts_default(&s->opts.opts);
    if (s->opts.opts.tol <= 0) ps_solve_opts_default(&s->opts.opts);
    if (s->opts.max_slots <= 0) s->opts.max_slots = 64;
    if (s->opts.epoch_iters <= 0) s->opts.epoch_iters = 64;
    std::memset(&s->st, 0, sizeof(s->st));
    if (cudaSetDevice(ctx->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete s;
        return PS_ECUDA;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return PS_OK;
}

extern "C" void ps_server_destroy(ps_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    std::lock_guard<std::mutex> ctx_lk(s->ctx->mu);
    cudaSetDevice(s->ctx->device);
    cudaStreamSynchronize(s->stream);
    batch_plan_free(s->plan);
    for (auto &kv : s->reqs) delete kv.second;
    for (auto &c : s->cases) dfree_all(s->ctx, c.allocs);
    cudaStreamDestroy(s->stream);
    delete s;
}

extern "C" int ps_server_add_case(ps_server *s, ps_mesh *mesh, const double *x0, int32_t *case_id) {
    if (!s || !mesh || !case_id || mesh->ctx != s->ctx) return PS_EINVAL;
    if (!mesh->coeff_ok) return PS_ESTATE;
    Case c;
    c.mesh = mesh;
    c.ws_bytes = batch_ws_bytes(mesh);
    c.single = s->opts.single_nodes > 0 && mesh->prep.n_nodes >= (int64_t)s->opts.single_nodes;
    const size_t bytes = (size_t)mesh->prep.n_nodes * 8;
    {
        std::lock_guard<std::mutex> ctx_lk(s->ctx->mu);
        cudaSetDevice(s->ctx->device);
        void *p = nullptr;
        int rc = dalloc(s->ctx, &p, bytes, c.allocs);
        c.b_dev = (double *)p;
        if (rc == PS_OK) rc = dalloc(s->ctx, &p, bytes, c.allocs), c.x_dev = (double *)p;
        if (rc == PS_OK)
            rc = dalloc(s->ctx, &p, (size_t)mesh->prep.n_elems * 8, c.allocs), c.beta_dev = (double *)p;
        if (rc == PS_OK) {
            cudaError_t e = x0 ? cudaMemcpy(c.x_dev, x0, bytes, cudaMemcpyHostToDevice) : cudaMemset(c.x_dev, 0, bytes);
            if (e == cudaSuccess) e = cudaMemset(c.b_dev, 0, bytes);
            if (e != cudaSuccess) rc = PS_ECUDA;
        }
        if (rc != PS_OK) {
            dfree_all(s->ctx, c.allocs);
            return rc;
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto &o : s->cases)
        if (o.mesh == mesh) {
            dfree_all(s->ctx, c.allocs);
            return PS_EINVAL;   // one case per mesh: its warm start lives on the device
        }
    s->cases.push_back(std::move(c));
    *case_id = (int32_t)s->cases.size() - 1;
    return PS_OK;
}

extern "C" int ps_solve_submit(ps_server *s, int32_t case_id, const double *b, const double *beta, ps_ticket *out) {
    if (!s || !b || !out) return PS_EINVAL;
    // the case's sizes (cases are only ever appended; their meshes fixed)
    int64_t n_nodes = 0, n_elems = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (case_id < 0 || case_id >= (int32_t)s->cases.size()) return PS_ENOTFOUND;
        n_nodes = s->cases[case_id].mesh->prep.n_nodes;
        n_elems = s->cases[case_id].mesh->prep.n_elems;
    }
    // validate and copy the inputs outside the lock (the worker keeps running)
    if (beta)
        for (int64_t e = 0; e < n_elems; ++e)
            if (!(beta[e] > 0.0) || !std::isfinite(beta[e])) return PS_EINVAL;
    Req *r = new (std::nothrow) Req();
    if (!r) return PS_ENOMEM;
    r->b.assign(b, b + n_nodes);
    if (beta) r->beta.assign(beta, beta + n_elems);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        Case &c = s->cases[case_id];
        r->id = s->next_ticket++;
        r->case_id = case_id;
        r->t_submit = now_s();
        std::memset(&r->info, 0, sizeof(r->info));
        c.queue.push_back(r);
        s->reqs[r->id] = r;
        s->st.submitted++;
        s->st.queued++;
        *out = r->id;
    }
    s->cv_work.notify_all();
    return PS_OK;
}

static int poll_locked(ps_server *s, ps_ticket t, ps_solve_info *info, double *x_out) {
    auto it = s->reqs.find(t);
    if (it == s->reqs.end()) return PS_ENOTFOUND;
    Req *r = it->second;
    if (r->status == PS_PENDING) return PS_PENDING;
    if (info) *info = r->info;
    if (x_out && !r->x.empty()) std::memcpy(x_out, r->x.data(), r->x.size() * 8);
    return r->status;
}

extern "C" int ps_solve_poll(ps_server *s, ps_ticket t, ps_solve_info *info, double *x_out) {
    if (!s) return PS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    return poll_locked(s, t, info, x_out);
}

extern "C" int ps_solve_wait(ps_server *s, ps_ticket t, double timeout_s, ps_solve_info *info, double *x_out) {
    if (!s) return PS_EINVAL;
    if (timeout_s <= 0) timeout_s = 600.0;
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    for (;;) {
        int st = poll_locked(s, t, info, x_out);
        if (st != PS_PENDING) return st;
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) return poll_locked(s, t, info, x_out);
    }
}

extern "C" int ps_server_release(ps_server *s, ps_ticket t) {
    if (!s) return PS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(t);
    if (it == s->reqs.end()) return PS_ENOTFOUND;
    if (it->second->status == PS_PENDING) return PS_ESTATE;
    delete it->second;
    s->reqs.erase(it);
    return PS_OK;
}

extern "C" int ps_server_get_stats(ps_server *s, ps_server_stats *out) {
    if (!s || !out) return PS_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->st;
    out->bytes_in_use = s->in_flight_bytes;
    return PS_OK;
}
