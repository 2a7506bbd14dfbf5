// Batched implicit FLD steps: many independent problems of uneven size in one
// persistent cooperative launch, captured once in a CUDA graph and replayed.
//
// Schedule.  Every problem gets a team of blocks sized to its cell count
// (ceil(N / cells_per_block), rounded down to a power of two, at most max_team and at
// most the problem's partial-sum capacity).  Problems with the same team size form a
// class; the co-resident grid is split between classes in proportion to their
// estimated work (cells x iterations of the previous step, or a size-based guess), and
// within a class the teams pull problems from a queue ordered by decreasing work
// (longest-processing-time first).  cells_per_block and max_team are the tunables the
// autotuner searches; its choice is cached per shape class of the batch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "gq_device.cuh"
#include "gq_internal.h"

namespace {

constexpr int kDefaultCellsPerBlock = 32768;
constexpr int kDefaultMaxTeam = 16;

std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune_cache;   // shape class -> (cells_per_block, max_team)

int pow2_floor(int v) {
    int p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}

}  // namespace

struct gq_batch {
    int n = 0;
    int cap = 0;             // problems the buffers can hold
    std::vector<gq_fld_plan*> plans;
    int device = 0;
    int grid_cap = 0;        // co-resident blocks of the batched solve kernel
    int grid = 0;            // blocks actually launched (sum of team sizes)
    int nteams = 0;
    int nclass = 0;
    int setup_total = 0;
    gq_batch_opts opts{};
    std::vector<double> est_iters;
    std::vector<int> prefix, block_team, team_first, team_size, team_class, queue, class_start;
    // device buffer
    void* dbuf = nullptr;
    gq::ProbDesc* d_desc = nullptr;
    int* d_ints = nullptr;      // prefix | block_team | team_first | team_size | team_class | queue | class_start
    int* d_state = nullptr;     // queue_head[n_class_cap] | team_slot[G] | abort
    unsigned* d_team_bar = nullptr;
    gq::SolveCtl* d_ctl_out = nullptr;
    size_t state_bytes = 0;
    // pinned host
    gq::ProbDesc* h_desc = nullptr;
    gq::SolveCtl* h_ctl_out = nullptr;
    gq::BatchArgs args{};
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
    cudaGraphExec_t gexec = nullptr;
    bool graph_failed = false;
    float last_ms = 0.f;
    long long spin = gq::kDefaultSpin;
};

namespace {

std::string shape_key(const gq_batch* B, const gq_batch_item* items) {
    // histogram of log2(cells) plus the precision mix
    int hist[40] = {0};
    int mixed = 0;
    long long cells = 0;
    for (int p = 0; p < B->n; p++) {
        const int N = B->plans[p]->N;
        cells += N;
        hist[std::min(39, (int)std::floor(std::log2((double)N)))]++;
        if (items && items[p].opts.prec == GQ_PREC_MIXED) mixed++;
    }
    std::string k = std::to_string(B->n) + ":" + std::to_string(mixed) + ":";
    for (int h : hist) k += std::to_string(h) + ",";
    return k;
}

// schedule from the current options and work estimates; returns false if it does not fit
bool build_schedule(gq_batch* B) {
    const int n = B->n;
    const int cpb = B->opts.cells_per_block > 0 ? B->opts.cells_per_block : kDefaultCellsPerBlock;
    const int maxt = B->opts.max_team > 0 ? B->opts.max_team : kDefaultMaxTeam;
    std::vector<int> tsize(n);
    std::vector<double> work(n);
    for (int p = 0; p < n; p++) {
        const gq_fld_plan* P = B->plans[p];
        int s = (int)std::min<long long>((P->N + (long long)cpb - 1) / cpb, 1ll << 20);
        s = std::max(1, std::min({s, maxt, P->solve_grid_max, B->grid_cap}));
        tsize[p] = pow2_floor(s);
        work[p] = (double)P->N * std::max(1.0, B->est_iters[p]);
    }
    std::vector<int> sizes(tsize);
    std::sort(sizes.begin(), sizes.end());
    sizes.erase(std::unique(sizes.begin(), sizes.end()), sizes.end());
    const int C = (int)sizes.size();
    std::vector<std::vector<int>> members(C);
    std::vector<double> cwork(C, 0.0);
    for (int p = 0; p < n; p++) {
        const int c = (int)(std::lower_bound(sizes.begin(), sizes.end(), tsize[p]) - sizes.begin());
        members[c].push_back(p);
        cwork[c] += work[p];
    }
    // teams per class: at least one, at most one per member, blocks in proportion to work
    const double wt = std::accumulate(cwork.begin(), cwork.end(), 0.0);
    std::vector<int> teams(C, 1);
    int used = 0;
    for (int c = 0; c < C; c++) used += sizes[c];
    if (used > B->grid_cap) return false;
    for (int c = 0; c < C; c++) {
        const int want = (int)std::floor((double)B->grid_cap * cwork[c] / wt / sizes[c]);
        const int add = std::max(0, std::min(want, (int)members[c].size()) - 1);
        const int room = (B->grid_cap - used) / sizes[c];
        const int a = std::min(add, room);
        teams[c] += a;
        used += a * sizes[c];
    }
    // leftover blocks: to the class with the most work per team
    while (true) {
        int best = -1;
        double bw = -1.0;
        for (int c = 0; c < C; c++) {
            if (teams[c] >= (int)members[c].size() || used + sizes[c] > B->grid_cap) continue;
            const double w = cwork[c] / teams[c];
            if (w > bw) { bw = w; best = c; }
        }
        if (best < 0) break;
        teams[best]++;
        used += sizes[best];
    }
    B->block_team.assign(used, 0);
    B->team_first.clear();
    B->team_size.clear();
    B->team_class.clear();
    int cursor = 0;
    for (int c = 0; c < C; c++)
        for (int t = 0; t < teams[c]; t++) {
            const int id = (int)B->team_first.size();
            B->team_first.push_back(cursor);
            B->team_size.push_back(sizes[c]);
            B->team_class.push_back(c);
            for (int b = 0; b < sizes[c]; b++) B->block_team[cursor + b] = id;
            cursor += sizes[c];
        }
    B->queue.clear();
    B->class_start.assign(1, 0);
    for (int c = 0; c < C; c++) {
        auto m = members[c];
        std::stable_sort(m.begin(), m.end(), [&](int a, int b) { return work[a] > work[b]; });
        B->queue.insert(B->queue.end(), m.begin(), m.end());
        B->class_start.push_back((int)B->queue.size());
    }
    B->grid = used;
    B->nteams = (int)B->team_first.size();
    B->nclass = C;
    return true;
}

cudaError_t upload_schedule(gq_batch* B) {
    const int n = B->cap, G = B->grid_cap;
    int* base = B->d_ints;
    std::vector<int> buf;
    auto put = [&](const std::vector<int>& v, size_t cap) {
        std::vector<int> t(v);
        t.resize(cap, 0);
        buf.insert(buf.end(), t.begin(), t.end());
    };
    put(B->prefix, n + 1);
    put(B->block_team, G);
    put(B->team_first, G);
    put(B->team_size, G);
    put(B->team_class, G);
    put(B->queue, n);
    put(B->class_start, G + 1);
    return cudaMemcpy(base, buf.data(), buf.size() * sizeof(int), cudaMemcpyHostToDevice);
}

void set_args(gq_batch* B) {
    const int n = B->cap, G = B->grid_cap;
    int* base = B->d_ints;
    gq::BatchArgs& a = B->args;
    a.desc = B->d_desc;
    a.n = B->n;
    a.nclass = B->nclass;
    a.setup_prefix = base;
    a.block_team = base + (n + 1);
    a.team_first = a.block_team + G;
    a.team_size = a.team_first + G;
    a.team_class = a.team_size + G;
    a.queue = a.team_class + G;
    a.class_start = a.queue + n;
    a.queue_head = B->d_state;
    a.team_slot = B->d_state + G;
    a.abort_flag = B->d_state + 2 * G;
    a.team_bar = B->d_team_bar;
    a.spin_limit = B->spin;
    a.ctl_out = B->d_ctl_out;
}

// the work of one batched step, enqueued on the batch stream (captured or eager)
cudaError_t enqueue_step(gq_batch* B) {
    cudaStream_t st = B->stream;
    cudaError_t e = cudaMemcpyAsync(B->d_desc, B->h_desc, sizeof(gq::ProbDesc) * B->n, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(B->d_state, 0, B->state_bytes, st);
    if (e == cudaSuccess) e = gq::launch_batch_setup(B->args, B->setup_total, st);
    if (e == cudaSuccess) e = gq::launch_batch_solve(B->args, B->grid, st);
    if (e == cudaSuccess) e = gq::launch_batch_finish(B->args, B->setup_total, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B->h_ctl_out, B->d_ctl_out, sizeof(gq::SolveCtl) * B->n, cudaMemcpyDeviceToHost, st);
    return e;
}

void drop_graph(gq_batch* B) {
    if (B->gexec) cudaGraphExecDestroy(B->gexec);
    B->gexec = nullptr;
}

cudaError_t run_step(gq_batch* B, cudaStream_t user) {
    cudaError_t e = cudaEventRecord(B->ev_in, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(B->stream, B->ev_in, 0);
    if (e != cudaSuccess) return e;
    const bool want_graph = B->opts.use_graph != 0 && !B->graph_failed;
    if (want_graph && !B->gexec) {
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e2 = enqueue_step(B);
            e = cudaStreamEndCapture(B->stream, &g);
            if (e2 != cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&B->gexec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            B->gexec = nullptr;
            B->graph_failed = true;
        }
    }
    e = cudaEventRecord(B->ev_t0, B->stream);
    if (e != cudaSuccess) return e;
    if (B->gexec) e = cudaGraphLaunch(B->gexec, B->stream);
    else e = enqueue_step(B);
    if (e == cudaSuccess) e = cudaEventRecord(B->ev_t1, B->stream);
    if (e == cudaSuccess) e = cudaEventRecord(B->ev_out, B->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, B->ev_out, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(B->stream);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&B->last_ms, B->ev_t0, B->ev_t1);
    return e;
}

gq_status fill_descs(gq_batch* B, const gq_batch_item* items) {
    for (int p = 0; p < B->n; p++) {
        const gq_batch_item& it = items[p];
        gq::ProbDesc& d = B->h_desc[p];
        const gq_fld_plan* P = B->plans[p];
        gq::StepParams sp{};
        gq::SolveParams pp{};
        gq_status s = gq::make_step_params(P, it.rho, it.e_g, it.E_r, it.T_g_out, &it.opacity, &it.eos, it.dt,
                                           &it.bc, &it.opts, &sp, &pp, nullptr);
        if (s != GQ_OK) return s;
        if (sp.eos_n != 0) return GQ_ERR_INVALID_ARG;   // batched steps take no EoS table
        sp.sadv = nullptr;   // batched steps take no explicit source
        sp.sig_n = sp.E_n = nullptr;
        d.sp = sp;
        d.g = P->geo;
        d.w = P->ws;
        d.solve = pp;
        d.setup_blocks = B->prefix[p + 1] - B->prefix[p];
        d.pad = 0;
        const_cast<gq_fld_plan*>(P)->last_precond = pp.precond;
    }
    return GQ_OK;
}

}  // namespace

namespace gq {

// A batch with buffers for up to `cap` problems and no members yet.
gq_status batch_create_capacity(int device, int num_sms, int cap, const gq_batch_opts* opts, gq_batch** out) {
    *out = nullptr;
    if (cap < 1) return GQ_ERR_INVALID_ARG;
    gq_batch* B = new (std::nothrow) gq_batch();
    if (!B) return GQ_ERR_OOM;
    B->cap = cap;
    B->device = device;
    if (opts) B->opts = *opts;
    else gq_batch_opts_default(&B->opts);
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != device) cudaSetDevice(device);
    auto fail = [&](gq_status s) {
        gq_batch_destroy(B);
        if (cur != device) cudaSetDevice(cur);
        return s;
    };
    const int per_sm = batch_solve_max_blocks_per_sm();
    if (per_sm < 1) return fail(GQ_ERR_CUDA);
    B->grid_cap = per_sm * num_sms;
    const int G = B->grid_cap;
    const size_t n_ints = (cap + 1) + 4 * (size_t)G + cap + (G + 1);
    B->state_bytes = sizeof(int) * (2 * (size_t)G + 1);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) & ~size_t(255);
        const size_t o = off;
        off += bytes;
        return o;
    };
    const size_t o_desc = take(sizeof(ProbDesc) * cap);
    const size_t o_ints = take(sizeof(int) * n_ints);
    const size_t o_state = take(B->state_bytes + sizeof(unsigned) * 2 * (size_t)G);
    const size_t o_ctl = take(sizeof(SolveCtl) * cap);
    if (cudaMalloc(&B->dbuf, off + 256) != cudaSuccess) {
        cudaGetLastError();
        return fail(GQ_ERR_OOM);
    }
    char* base = static_cast<char*>(B->dbuf);
    B->d_desc = reinterpret_cast<ProbDesc*>(base + o_desc);
    B->d_ints = reinterpret_cast<int*>(base + o_ints);
    B->d_state = reinterpret_cast<int*>(base + o_state);
    B->d_team_bar = reinterpret_cast<unsigned*>(base + o_state + B->state_bytes);
    B->state_bytes += sizeof(unsigned) * 2 * (size_t)G;   // barriers are reset with the state
    B->d_ctl_out = reinterpret_cast<SolveCtl*>(base + o_ctl);
    if (cudaMallocHost(reinterpret_cast<void**>(&B->h_desc), sizeof(ProbDesc) * cap) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&B->h_ctl_out), sizeof(SolveCtl) * cap) != cudaSuccess) {
        cudaGetLastError();
        return fail(GQ_ERR_OOM);
    }
    std::memset(B->h_desc, 0, sizeof(ProbDesc) * cap);
    if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&B->ev_t0) != cudaSuccess || cudaEventCreate(&B->ev_t1) != cudaSuccess)
        return fail(GQ_ERR_CUDA);
    if (cur != device) cudaSetDevice(cur);
    *out = B;
    return GQ_OK;
}

// Make plans[0..n) the members (n <= cap), rebuild and upload the schedule.
gq_status batch_rebind(gq_batch* B, gq_fld_plan* const* plans, int n) {
    if (!B || n < 1 || n > B->cap) return GQ_ERR_INVALID_ARG;
    for (int p = 0; p < n; p++)
        if (!plans[p] || plans[p]->device != B->device) return GQ_ERR_INVALID_ARG;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != B->device) cudaSetDevice(B->device);
    if (B->stream) cudaStreamSynchronize(B->stream);
    const bool same = n == B->n && std::equal(plans, plans + n, B->plans.begin());
    std::vector<double> est(n);
    for (int p = 0; p < n; p++) {
        // keep the measured iteration count of a plan that stays in the batch
        double e = 20.0 + 2.0 * std::sqrt((double)plans[p]->N);
        for (int q = 0; q < B->n; q++)
            if (B->plans[q] == plans[p]) e = B->est_iters[q];
        est[p] = e;
    }
    B->n = n;
    B->plans.assign(plans, plans + n);
    B->est_iters = est;
    B->prefix.assign(n + 1, 0);
    for (int p = 0; p < n; p++) B->prefix[p + 1] = B->prefix[p] + plans[p]->setup_blocks;
    B->setup_total = B->prefix[n];
    if (!same && (B->opts.cells_per_block <= 0 || B->opts.max_team <= 0)) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(shape_key(B, nullptr));
        if (it != g_tune_cache.end()) {
            if (B->opts.cells_per_block <= 0) B->opts.cells_per_block = it->second.first;
            if (B->opts.max_team <= 0) B->opts.max_team = it->second.second;
        }
    }
    gq_status st = GQ_OK;
    if (!build_schedule(B)) st = GQ_ERR_INVALID_ARG;
    else if (upload_schedule(B) != cudaSuccess) st = GQ_ERR_CUDA;
    set_args(B);
    drop_graph(B);
    if (cur != B->device) cudaSetDevice(cur);
    return st;
}

}  // namespace gq

extern "C" {

void gq_batch_opts_default(gq_batch_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->cells_per_block = 0;
    o->max_team = 0;
    o->use_graph = 1;
}

gq_status gq_batch_create(gq_fld_plan* const* plans, int n, const gq_batch_opts* opts, gq_batch** out) {
    if (!out) return GQ_ERR_INVALID_ARG;
    *out = nullptr;
    if (!plans || n < 1) return GQ_ERR_INVALID_ARG;
    for (int p = 0; p < n; p++)
        if (!plans[p]) return GQ_ERR_INVALID_ARG;
    gq_batch* B = nullptr;
    gq_status s = gq::batch_create_capacity(plans[0]->device, plans[0]->num_sms, n, opts, &B);
    if (s != GQ_OK) return s;
    s = gq::batch_rebind(B, plans, n);
    if (s != GQ_OK) {
        gq_batch_destroy(B);
        return s;
    }
    *out = B;
    return GQ_OK;
}

gq_status gq_batch_step(gq_batch* B, const gq_batch_item* items, void* stream, gq_step_info* infos) {
    if (!B || !items) return GQ_ERR_INVALID_ARG;
    if (infos) std::memset(infos, 0, sizeof(gq_step_info) * B->n);
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess) return GQ_ERR_CUDA;
    if (cur != B->device && cudaSetDevice(B->device) != cudaSuccess) return GQ_ERR_CUDA;
    gq_status vs = fill_descs(B, items);
    if (vs != GQ_OK) {
        if (cur != B->device) cudaSetDevice(cur);
        return vs;
    }
    long long spin = 0;
    for (int p = 0; p < B->n; p++) spin = std::max(spin, (long long)B->h_desc[p].solve.spin_limit);
    if (spin != B->spin) {
        B->spin = spin;
        set_args(B);
        drop_graph(B);
    }
    cudaError_t e = run_step(B, static_cast<cudaStream_t>(stream));
    if (cur != B->device) cudaSetDevice(cur);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return GQ_ERR_CUDA;
    }
    gq_status worst = GQ_OK;
    for (int p = 0; p < B->n; p++) {
        const gq::SolveCtl& c = B->h_ctl_out[p];
        const gq_status s = gq::status_of(c);
        if (infos) {
            gq::fill_info(c, s, &infos[p]);
            infos[p].t_solve_ms = B->last_ms;
        }
        if (c.iterations > 0) B->est_iters[p] = c.iterations;
        if (s != GQ_OK && worst == GQ_OK) worst = s;
    }
    return worst;
}

gq_status gq_batch_reschedule(gq_batch* B, const gq_batch_opts* opts) {
    if (!B) return GQ_ERR_INVALID_ARG;
    if (opts) {
        B->opts.cells_per_block = opts->cells_per_block;
        B->opts.max_team = opts->max_team;
        if (opts->use_graph != B->opts.use_graph) drop_graph(B);
        B->opts.use_graph = opts->use_graph;
    }
    const int old_grid = B->grid;
    if (!build_schedule(B)) return GQ_ERR_INVALID_ARG;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != B->device) cudaSetDevice(B->device);
    cudaError_t e = cudaStreamSynchronize(B->stream);
    if (e == cudaSuccess) e = upload_schedule(B);
    set_args(B);
    if (B->grid != old_grid || B->args.nclass != B->nclass) drop_graph(B);
    drop_graph(B);   // kernel arguments (class count, grid) are baked into the graph
    if (cur != B->device) cudaSetDevice(cur);
    return e == cudaSuccess ? GQ_OK : GQ_ERR_CUDA;
}

gq_status gq_batch_autotune(gq_batch* B, const gq_batch_item* items, void* stream, gq_batch_opts* best_out,
                            double* best_ms_out) {
    if (!B || !items) return GQ_ERR_INVALID_ARG;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != B->device) cudaSetDevice(B->device);
    // the steps below overwrite e_g and E_r: keep a copy of the inputs and restore them
    size_t total = 0;
    for (int p = 0; p < B->n; p++) total += (size_t)B->plans[p]->N;
    double* save = nullptr;
    if (cudaMalloc(&save, 2 * total * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        if (cur != B->device) cudaSetDevice(cur);
        return GQ_ERR_OOM;
    }
    cudaStream_t us = static_cast<cudaStream_t>(stream);
    auto copy_all = [&](bool to_save) {
        size_t o = 0;
        cudaError_t e = cudaSuccess;
        for (int p = 0; p < B->n && e == cudaSuccess; p++) {
            const size_t N = (size_t)B->plans[p]->N;
            double* s0 = save + o;
            double* s1 = save + total + o;
            if (to_save) {
                e = cudaMemcpyAsync(s0, items[p].e_g, N * sizeof(double), cudaMemcpyDeviceToDevice, us);
                if (e == cudaSuccess) e = cudaMemcpyAsync(s1, items[p].E_r, N * sizeof(double), cudaMemcpyDeviceToDevice, us);
            } else {
                e = cudaMemcpyAsync(items[p].e_g, s0, N * sizeof(double), cudaMemcpyDeviceToDevice, us);
                if (e == cudaSuccess) e = cudaMemcpyAsync(items[p].E_r, s1, N * sizeof(double), cudaMemcpyDeviceToDevice, us);
            }
            o += N;
        }
        return e;
    };
    gq_status result = GQ_OK;
    gq_batch_opts best = B->opts;
    double best_ms = 1e300;
    if (copy_all(true) != cudaSuccess) result = GQ_ERR_CUDA;
    // one step first, for the per-problem iteration estimates
    if (result == GQ_OK) {
        gq_status s = gq_batch_step(B, items, stream, nullptr);
        if (s == GQ_ERR_CUDA) result = s;
    }
    const int cpbs[] = {8192, 16384, 32768, 65536, 131072};
    const int teams[] = {4, 8, 16, 32};
    for (int cpb : cpbs) {
        for (int mt : teams) {
            if (result != GQ_OK) break;
            gq_batch_opts o = B->opts;
            o.cells_per_block = cpb;
            o.max_team = mt;
            if (gq_batch_reschedule(B, &o) != GQ_OK) continue;
            if (copy_all(false) != cudaSuccess) { result = GQ_ERR_CUDA; break; }
            gq_status s = gq_batch_step(B, items, stream, nullptr);   // graph capture + first replay
            if (s == GQ_ERR_CUDA) { result = s; break; }
            if (copy_all(false) != cudaSuccess) { result = GQ_ERR_CUDA; break; }
            s = gq_batch_step(B, items, stream, nullptr);
            if (s == GQ_ERR_CUDA) { result = s; break; }
            if (B->last_ms < best_ms) {
                best_ms = B->last_ms;
                best = B->opts;
            }
        }
    }
    if (copy_all(false) != cudaSuccess && result == GQ_OK) result = GQ_ERR_CUDA;
    cudaStreamSynchronize(us);
    cudaFree(save);
    if (result == GQ_OK) {
        gq_batch_reschedule(B, &best);
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[shape_key(B, items)] = {best.cells_per_block, best.max_team};
        g_tune_cache[shape_key(B, nullptr)] = {best.cells_per_block, best.max_team};
    }
    if (best_out) *best_out = best;
    if (best_ms_out) *best_ms_out = best_ms;
    if (cur != B->device) cudaSetDevice(cur);
    return result;
}

double gq_batch_last_step_ms(const gq_batch* B) { return B ? (double)B->last_ms : 0.0; }

int gq_batch_uses_graph(const gq_batch* B) { return (B && B->gexec) ? 1 : 0; }

void gq_batch_destroy(gq_batch* B) {
    if (!B) return;
    if (B->stream) cudaStreamSynchronize(B->stream);
    drop_graph(B);
    if (B->dbuf) cudaFree(B->dbuf);
    if (B->h_desc) cudaFreeHost(B->h_desc);
    if (B->h_ctl_out) cudaFreeHost(B->h_ctl_out);
    if (B->ev_in) cudaEventDestroy(B->ev_in);
    if (B->ev_out) cudaEventDestroy(B->ev_out);
    if (B->ev_t0) cudaEventDestroy(B->ev_t0);
    if (B->ev_t1) cudaEventDestroy(B->ev_t1);
    if (B->stream) cudaStreamDestroy(B->stream);
    delete B;
}

gq_status gq_fld_step_batched(gq_fld_plan* const* plans, int n, const gq_batch_item* items, void* stream,
                              gq_step_info* infos) {
    gq_batch_opts o;
    gq_batch_opts_default(&o);
    o.use_graph = 0;
    gq_batch* B = nullptr;
    gq_status s = gq_batch_create(plans, n, &o, &B);
    if (s != GQ_OK) return s;
    s = gq_batch_step(B, items, stream, infos);
    gq_batch_destroy(B);
    return s;
}

}  // extern "C"
