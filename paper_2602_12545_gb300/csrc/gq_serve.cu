// Continuous-batching server for implicit FLD solves.
//
// Requests (a grid, initial fields and a number of consecutive implicit steps) are
// queued with host copies of their inputs.  Each engine tick (gq_server_poll):
//   1. admits queued requests in arrival order while their device footprint (plan
//      arena plus rho, e_g, E_r, T_g) fits the memory budget and the active-set cap;
//      admission builds the plan and uploads the fields, which then stay resident;
//   2. steps every resident request once: the smaller ones together in one batched
//      persistent launch, so work from requests that arrived at different times overlaps
//      on the device, then each request of at least solo_cells cells alone on the whole
//      GPU (a batch team is capped at a few blocks, which would leave a large grid
//      running on a fraction of the SMs while the small ones finish);
//   3. retires requests that finished their steps (or failed): results are copied to the
//      caller's host buffers and their device memory is returned to the budget.
// The paper has no counterpart (its code advances one simulation per MPI job).
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "gq_device.cuh"
#include "gq_internal.h"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct ServeReq {
    int64_t id = 0;
    int nx = 0, ny = 0, coord = 0;
    std::vector<double> xf, yf, ax, ay, vol;
    std::vector<double> rho, eg, E;
    gq_opacity_law op{};
    gq_eos eos{};
    double dt = 0.0;
    gq_bc bc{};
    gq_solver_opts opts{};
    int n_steps = 0;
    double *E_out = nullptr, *eg_out = nullptr, *T_out = nullptr;
    // state
    int state = 0;              // 0 queued, 1 resident, 2 done
    gq_status status = GQ_OK;
    int steps_done = 0;
    int iterations = 0;
    gq_fld_plan* plan = nullptr;
    double* dfields = nullptr;  // rho | e_g | E_r | T_g
    size_t bytes = 0;
    double submit_s = 0.0, admit_s = 0.0, done_s = 0.0;
    double energy_before = 0.0, energy_after = 0.0;
};

}  // namespace

struct gq_server {
    gq_server_opts opts{};
    int device = 0;
    size_t used = 0;
    int64_t next_id = 1;
    std::deque<ServeReq*> queue;
    std::vector<ServeReq*> active;
    std::unordered_map<int64_t, ServeReq*> all;
    gq_batch* batch = nullptr;
    std::vector<gq_fld_plan*> bound;
    std::vector<gq_batch_item> items;
    std::vector<gq_step_info> infos;
    cudaStream_t stream = nullptr;
    std::mutex mu;
};

namespace {

size_t field_bytes(int nx, int ny) { return 4 * sizeof(double) * (size_t)nx * ny; }

gq_status admit(gq_server* S, ServeReq* R) {
    gq_grid_desc g{};
    g.nx = R->nx;
    g.ny = R->ny;
    g.coord = R->coord;
    g.x_faces = R->xf.data();
    g.y_faces = R->yf.data();
    g.area_x = R->ax.empty() ? nullptr : R->ax.data();
    g.area_y = R->ay.empty() ? nullptr : R->ay.data();
    g.volume = R->vol.empty() ? nullptr : R->vol.data();
    gq_status st = gq_fld_setup(&g, &R->plan);
    if (st != GQ_OK) return st;
    const size_t N = (size_t)R->nx * R->ny;
    if (cudaMalloc(&R->dfields, field_bytes(R->nx, R->ny)) != cudaSuccess) {
        cudaGetLastError();
        gq_fld_destroy(R->plan);
        R->plan = nullptr;
        return GQ_ERR_OOM;
    }
    cudaError_t e = cudaMemcpyAsync(R->dfields, R->rho.data(), N * sizeof(double), cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(R->dfields + N, R->eg.data(), N * sizeof(double), cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(R->dfields + 2 * N, R->E.data(), N * sizeof(double), cudaMemcpyHostToDevice, S->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(S->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(R->dfields);
        R->dfields = nullptr;
        gq_fld_destroy(R->plan);
        R->plan = nullptr;
        return GQ_ERR_CUDA;
    }
    // the host copies are no longer needed
    std::vector<double>().swap(R->rho);
    std::vector<double>().swap(R->eg);
    std::vector<double>().swap(R->E);
    R->bytes = gq_fld_plan_bytes(R->plan) + field_bytes(R->nx, R->ny);
    R->state = 1;
    R->admit_s = now_s();
    return GQ_OK;
}

void retire(gq_server* S, ServeReq* R) {
    const size_t N = (size_t)R->nx * R->ny;
    if (R->dfields && (R->status == GQ_OK || R->status == GQ_ERR_NOT_CONVERGED)) {
        if (R->E_out) cudaMemcpy(R->E_out, R->dfields + 2 * N, N * sizeof(double), cudaMemcpyDeviceToHost);
        if (R->eg_out) cudaMemcpy(R->eg_out, R->dfields + N, N * sizeof(double), cudaMemcpyDeviceToHost);
        if (R->T_out) cudaMemcpy(R->T_out, R->dfields + 3 * N, N * sizeof(double), cudaMemcpyDeviceToHost);
    }
    if (R->dfields) cudaFree(R->dfields);
    R->dfields = nullptr;
    if (R->plan) gq_fld_destroy(R->plan);
    R->plan = nullptr;
    if (S->used >= R->bytes) S->used -= R->bytes;
    else S->used = 0;
    R->state = 2;
    R->done_s = now_s();
}

}  // namespace

extern "C" {

size_t gq_server_request_bytes(int nx, int ny) {
    const size_t plan = gq_fld_plan_bytes_for(nx, ny);
    return plan ? plan + field_bytes(nx, ny) : 0;
}

gq_status gq_server_create(const gq_server_opts* opts, gq_server** out) {
    if (!out) return GQ_ERR_INVALID_ARG;
    *out = nullptr;
    if (!opts || opts->budget_bytes == 0 || opts->max_active < 0) return GQ_ERR_INVALID_ARG;
    gq_server* S = new (std::nothrow) gq_server();
    if (!S) return GQ_ERR_OOM;
    S->opts = *opts;
    if (S->opts.max_active == 0) S->opts.max_active = 256;
    if (S->opts.solo_cells == 0) S->opts.solo_cells = 1 << 19;
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return GQ_ERR_CUDA;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S->device);
    gq_batch_opts bo;
    gq_batch_opts_default(&bo);
    bo.use_graph = S->opts.use_graph;
    gq_status st = gq::batch_create_capacity(S->device, sms, S->opts.max_active, &bo, &S->batch);
    if (st != GQ_OK) {
        delete S;
        return st;
    }
    if (cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking) != cudaSuccess) {
        gq_batch_destroy(S->batch);
        delete S;
        return GQ_ERR_CUDA;
    }
    *out = S;
    return GQ_OK;
}

gq_status gq_server_submit(gq_server* S, const gq_request* rq, int64_t* id_out) {
    if (rq && rq->eos.table_n != 0) return GQ_ERR_INVALID_ARG;   // requests take no EoS table
    if (!S || !rq || !id_out) return GQ_ERR_INVALID_ARG;
    const gq_grid_desc& g = rq->grid;
    if (g.nx < 1 || g.ny < 1 || !g.x_faces || !g.y_faces || !rq->rho || !rq->e_g || !rq->E_r || rq->n_steps < 1)
        return GQ_ERR_INVALID_ARG;
    if ((long long)g.nx * g.ny > gq::kMaxCells) return GQ_ERR_INVALID_ARG;
    const size_t need = gq_server_request_bytes(g.nx, g.ny);
    if (need == 0) return GQ_ERR_CUDA;
    if (need > S->opts.budget_bytes) return GQ_ERR_BUDGET;
    ServeReq* R = new (std::nothrow) ServeReq();
    if (!R) return GQ_ERR_OOM;
    const size_t N = (size_t)g.nx * g.ny;
    R->nx = g.nx;
    R->ny = g.ny;
    R->coord = g.coord;
    R->xf.assign(g.x_faces, g.x_faces + g.nx + 1);
    R->yf.assign(g.y_faces, g.y_faces + g.ny + 1);
    if (g.area_x) R->ax.assign(g.area_x, g.area_x + (size_t)g.ny * (g.nx + 1));
    if (g.area_y) R->ay.assign(g.area_y, g.area_y + (size_t)(g.ny + 1) * g.nx);
    if (g.volume) R->vol.assign(g.volume, g.volume + N);
    R->rho.assign(rq->rho, rq->rho + N);
    R->eg.assign(rq->e_g, rq->e_g + N);
    R->E.assign(rq->E_r, rq->E_r + N);
    R->op = rq->opacity;
    R->eos = rq->eos;
    R->dt = rq->dt;
    R->bc = rq->bc;
    R->opts = rq->opts;
    R->n_steps = rq->n_steps;
    R->E_out = rq->E_r_out;
    R->eg_out = rq->e_g_out;
    R->T_out = rq->T_g_out;
    R->submit_s = now_s();
    std::lock_guard<std::mutex> lk(S->mu);
    R->id = S->next_id++;
    S->queue.push_back(R);
    S->all[R->id] = R;
    *id_out = R->id;
    return GQ_OK;
}

gq_status gq_server_poll(gq_server* S, int* completed) {
    if (!S) return GQ_ERR_INVALID_ARG;
    if (completed) *completed = 0;
    std::lock_guard<std::mutex> lk(S->mu);
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != S->device) cudaSetDevice(S->device);
    int done = 0;
    // 1. admission (arrival order, budget and active-set cap)
    while (!S->queue.empty() && (int)S->active.size() < S->opts.max_active) {
        ServeReq* R = S->queue.front();
        const size_t need = gq_server_request_bytes(R->nx, R->ny);
        if (S->used + need > S->opts.budget_bytes) break;
        S->queue.pop_front();
        gq_status st = admit(S, R);
        if (st != GQ_OK) {
            R->status = st;
            retire(S, R);
            done++;
            continue;
        }
        S->used += R->bytes;
        S->active.push_back(R);
    }
    if (S->active.empty()) {
        if (cur != S->device) cudaSetDevice(cur);
        if (completed) *completed = done;
        return GQ_OK;
    }
    // 2. one step of every resident request: the small ones in one batched launch, the
    //    large ones (at least solo_cells cells) each alone on the whole GPU
    const int n = (int)S->active.size();
    S->infos.assign(n, gq_step_info{});
    std::vector<int> small, large;
    for (int p = 0; p < n; p++) {
        const ServeReq* R = S->active[p];
        const long long cells = (long long)R->nx * R->ny;
        (S->opts.solo_cells > 0 && cells >= S->opts.solo_cells ? large : small).push_back(p);
    }
    gq_status bst = GQ_OK;
    if (!small.empty()) {
        const int m = (int)small.size();
        std::vector<gq_fld_plan*> plans(m);
        for (int i = 0; i < m; i++) plans[i] = S->active[small[i]]->plan;
        if (plans != S->bound) {
            gq_status st = gq::batch_rebind(S->batch, plans.data(), m);
            if (st != GQ_OK) {
                if (cur != S->device) cudaSetDevice(cur);
                return st;
            }
            S->bound = plans;
        }
        S->items.assign(m, gq_batch_item{});
        std::vector<gq_step_info> binfo(m);
        for (int i = 0; i < m; i++) {
            ServeReq* R = S->active[small[i]];
            const size_t N = (size_t)R->nx * R->ny;
            gq_batch_item& it = S->items[i];
            it.rho = R->dfields;
            it.e_g = R->dfields + N;
            it.E_r = R->dfields + 2 * N;
            it.T_g_out = R->dfields + 3 * N;
            it.opacity = R->op;
            it.eos = R->eos;
            it.dt = R->dt;
            it.bc = R->bc;
            it.opts = R->opts;
        }
        bst = gq_batch_step(S->batch, S->items.data(), S->stream, binfo.data());
        for (int i = 0; i < m; i++) S->infos[small[i]] = binfo[i];
    }
    if (bst == GQ_ERR_CUDA || bst == GQ_ERR_INVALID_ARG) {
        // nothing ran: fail every resident request rather than retry forever
        for (ServeReq* R : S->active) {
            R->status = bst;
            retire(S, R);
            done++;
        }
        S->active.clear();
        S->bound.clear();
        if (cur != S->device) cudaSetDevice(cur);
        if (completed) *completed = done;
        return bst;
    }
    for (int p : large) {
        ServeReq* R = S->active[p];
        const size_t N = (size_t)R->nx * R->ny;
        gq_fld_step(R->plan, R->dfields, R->dfields + N, R->dfields + 2 * N, R->dfields + 3 * N, &R->op, &R->eos,
                    R->dt, &R->bc, &R->opts, S->stream, &S->infos[p]);
    }
    // 3. retire finished or failed requests
    std::vector<ServeReq*> keep;
    keep.reserve(n);
    for (int p = 0; p < n; p++) {
        ServeReq* R = S->active[p];
        const gq_step_info& inf = S->infos[p];
        if (R->steps_done == 0) R->energy_before = inf.energy_before;
        R->energy_after = inf.energy_after;
        R->steps_done++;
        R->iterations += inf.iterations;
        const gq_status st = static_cast<gq_status>(inf.status);
        if (st != GQ_OK) R->status = st;
        const bool failed = st != GQ_OK && st != GQ_ERR_NOT_CONVERGED;
        if (failed || R->steps_done >= R->n_steps) {
            retire(S, R);
            done++;
        } else {
            keep.push_back(R);
        }
    }
    S->active.swap(keep);
    if (cur != S->device) cudaSetDevice(cur);
    if (completed) *completed = done;
    return GQ_OK;
}

gq_status gq_server_info(gq_server* S, int64_t id, gq_request_info* out) {
    if (!S || !out) return GQ_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return GQ_ERR_INVALID_ARG;
    const ServeReq* R = it->second;
    std::memset(out, 0, sizeof(*out));
    out->state = R->state;
    out->status = R->status;
    out->steps_done = R->steps_done;
    out->iterations = R->iterations;
    out->submit_s = R->submit_s;
    out->admit_s = R->admit_s;
    out->done_s = R->done_s;
    out->energy_before = R->energy_before;
    out->energy_after = R->energy_after;
    out->device_bytes = R->bytes;
    return GQ_OK;
}

gq_status gq_server_release(gq_server* S, int64_t id) {
    if (!S) return GQ_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end() || it->second->state != 2) return GQ_ERR_INVALID_ARG;
    delete it->second;
    S->all.erase(it);
    return GQ_OK;
}

int gq_server_pending(gq_server* S) {
    if (!S) return 0;
    std::lock_guard<std::mutex> lk(S->mu);
    return (int)(S->queue.size() + S->active.size());
}

size_t gq_server_used_bytes(gq_server* S) {
    if (!S) return 0;
    std::lock_guard<std::mutex> lk(S->mu);
    return S->used;
}

void gq_server_destroy(gq_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (ServeReq* R : S->active) {
            if (R->dfields) cudaFree(R->dfields);
            if (R->plan) gq_fld_destroy(R->plan);
        }
        for (auto& kv : S->all) delete kv.second;
        S->all.clear();
        if (S->batch) gq_batch_destroy(S->batch);
        if (S->stream) cudaStreamDestroy(S->stream);
    }
    delete S;
}

}  // extern "C"
