// nks_server.cu -- request loop for many simulations on one GPU (serving).
//
// Requests (a grid, initial fields and a number of time steps) are grouped by
// grid shape.  Each shape group owns one batch (nks_create_batch) with a fixed
// number of slots, a CUDA stream and a worker thread.  Continuous batching:
// between two batch steps the worker loads newly admitted requests into free
// slots, steps every occupied slot once (one launch per solver phase for the
// whole group), and retires the requests that reached their step count, which
// frees their slots for the next arrivals.  Groups of different shapes run
// concurrently on their own streams, so their kernels overlap on the device.
// Admission is by device memory: a new group reserves slots x (bytes of one
// slot, measured on a one-slot batch of that shape) out of the server's
// budget; a group whose slots all emptied with nothing queued frees its
// memory.  Every result is bitwise the result of the same request run alone,
// because each batch slot performs exactly its own solver's work.
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "nks_internal.cuh"

using nks::set_thread_error;

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    long long id = 0;
    nks_grid grid{};
    std::vector<double> c, eta;
    int steps = 0;
    double t_submit = 0.0, t_admit = -1.0, t_done = -1.0;
    // outcome
    int status = NKS_OK;
    int steps_done = 0, newton_its = 0, gmres_its = 0, retries = 0;
    double t = 0.0, energy = 0.0, mass = 0.0;
    std::vector<double> u;
    std::string err;
    bool done = false;
};

struct ShapeKey {
    int dim, n0, n1, n2, bc;
    bool operator<(const ShapeKey &o) const
    {
        return std::tie(dim, n0, n1, n2, bc) < std::tie(o.dim, o.n0, o.n1, o.n2, o.bc);
    }
};

struct Group {
    ShapeKey key{};
    int slots = 0;
    size_t bytes = 0;                           // reserved device bytes
    std::deque<std::shared_ptr<Request>> queue; // admitted, not yet loaded
    int occupied = 0;                           // loaded + queued
    std::thread worker;
    bool finished = false;
};

void *stream_alloc(size_t bytes, void *ctx)
{
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, *(cudaStream_t *)ctx) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void stream_free(void *p, void *ctx) { cudaFreeAsync(p, *(cudaStream_t *)ctx); }

}  // namespace

struct nks_server {
    nks_coeffs coeffs{};
    nks_server_opts so{};
    int device = 0;
    Clock::time_point t0;
    std::mutex mu;
    std::condition_variable cv;
    long long next_id = 1;
    size_t used = 0;
    bool stopping = false;
    std::deque<std::shared_ptr<Request>> waiting;
    std::map<long long, std::shared_ptr<Request>> all;
    std::map<ShapeKey, std::unique_ptr<Group>> groups;
    std::vector<std::unique_ptr<Group>> retired;  // finished groups whose threads are joined later
    std::map<ShapeKey, size_t> slot_bytes;        // measured bytes of one slot per shape
    std::string err;

    double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

ShapeKey key_of(const nks_grid &g)
{
    return ShapeKey{g.dim, g.n[0], g.dim >= 2 ? g.n[1] : 1, g.dim == 3 ? g.n[2] : 1, g.bc};
}

nks_opts opts_for(const nks_server *S, const nks_grid &g)
{
    nks_opts o = S->so.opts;
    const int side = g.dim == 3 ? S->so.box_side_3d : (g.dim == 2 ? S->so.box_side_2d : 4 * S->so.box_side_2d);
    for (int J = 0; J < 3; J++) o.sub[J] = J < g.dim ? std::max(2, (g.n[J] + side / 2) / side) : 1;
    o.timing = 0;
    return o;
}

// bytes of one slot of this shape (a one-slot batch without fields); 0 on failure
size_t measure_slot(nks_server *S, const nks_grid &g)
{
    const nks_opts o = opts_for(S, g);
    nks_problem *H = nullptr;
    size_t b = 0;
    if (nks_create_batch(&g, 1, nullptr, nullptr, &S->coeffs, &o, nullptr, nullptr, &H) == NKS_OK) {
        b = nks_device_bytes(H);
        nks_destroy(H);
    }
    return b;
}

void finish(nks_server *S, const std::shared_ptr<Request> &r)
{
    r->t_done = S->now();
    r->done = true;
}

void worker_main(nks_server *S, Group *G);

// move waiting requests into groups while memory and group count allow (lock held)
void admit_locked(nks_server *S)
{
    for (auto it = S->waiting.begin(); it != S->waiting.end();) {
        std::shared_ptr<Request> r = *it;
        const ShapeKey k = key_of(r->grid);
        auto g = S->groups.find(k);
        if (g != S->groups.end() && !g->second->finished) {
            Group *G = g->second.get();
            if (G->occupied < G->slots) {
                G->queue.push_back(r);
                G->occupied++;
                it = S->waiting.erase(it);
                continue;
            }
            ++it;
            continue;
        }
        if ((int)S->groups.size() >= S->so.max_groups) {
            ++it;
            continue;
        }
        size_t per = S->slot_bytes[k];
        if (per == 0) {
            ++it;  // not measured yet (measured outside the lock by submit)
            continue;
        }
        const size_t room = S->so.mem_budget > S->used ? S->so.mem_budget - S->used : 0;
        const int fit = (int)std::min<size_t>((size_t)S->so.max_slots, room / per);
        if (fit < 1) {
            ++it;
            continue;
        }
        std::unique_ptr<Group> G(new Group());
        G->key = k;
        G->slots = fit;
        G->bytes = (size_t)fit * per;
        S->used += G->bytes;
        G->queue.push_back(r);
        G->occupied = 1;
        Group *gp = G.get();
        S->groups[k] = std::move(G);
        gp->worker = std::thread(worker_main, S, gp);
        it = S->waiting.erase(it);
    }
}

void worker_main(nks_server *S, Group *G)
{
    cudaSetDevice(S->device);
    cudaStream_t stream = nullptr;
    cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking);
    nks_allocator alloc{stream_alloc, stream_free, &stream};
    nks_grid grid{};
    {
        std::lock_guard<std::mutex> lk(S->mu);
        grid = G->queue.front()->grid;
    }
    const nks_opts o = opts_for(S, grid);
    nks_problem *B = nullptr;
    const int rc0 = nks_create_batch(&grid, G->slots, nullptr, nullptr, &S->coeffs, &o, &alloc, stream, &B);
    std::vector<std::shared_ptr<Request>> slot(G->slots);
    std::vector<nks_step_info> infos(G->slots);
    for (;;) {
        std::vector<std::shared_ptr<Request>> incoming;
        bool idle = false;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            int loaded = 0;
            for (auto &q : slot) loaded += q ? 1 : 0;
            if (rc0 != NKS_OK) {
                // the batch could not be created: fail everything routed here
                for (auto &q : G->queue) {
                    q->status = rc0;
                    q->err = "serving: batch creation failed";
                    finish(S, q);
                }
                G->occupied -= (int)G->queue.size();
                G->queue.clear();
                S->cv.notify_all();
            }
            if (loaded == 0 && G->queue.empty()) {
                // idle: leave the group table; the memory is returned below
                G->finished = true;
                auto self = S->groups.find(G->key);
                if (self != S->groups.end() && self->second.get() == G) {
                    S->retired.push_back(std::move(self->second));
                    S->groups.erase(self);
                }
                idle = true;
            }
            while (!idle && !G->queue.empty()) {
                incoming.push_back(G->queue.front());
                G->queue.pop_front();
            }
        }
        if (idle) break;
        // continuous batching: new requests take free slots at this step boundary
        std::vector<std::shared_ptr<Request>> failed;
        for (auto &r : incoming) {
            int s = 0;
            while (slot[s]) s++;
            r->t_admit = S->now();
            const int rc = nks_batch_load(B, s, r->c.data(), r->eta.data());
            if (rc != NKS_OK) {
                r->status = rc;
                r->err = nks_last_error(B);
                failed.push_back(r);
                continue;
            }
            slot[s] = r;
        }
        std::vector<int> retiring;
        bool any = false;
        for (auto &q : slot) any = any || q;
        if (any) {
            const int rc = nks_batch_step(B, nullptr, nullptr, infos.data());
            for (int s = 0; s < G->slots; s++) {
                Request *r = slot[s].get();
                if (!r) continue;
                const nks_step_info &f = infos[s];
                bool retire = false;
                if (rc != NKS_OK || f.status != NKS_OK) {
                    r->status = rc != NKS_OK ? rc : f.status;
                    r->err = nks_last_error(B);
                    retire = true;
                } else {
                    r->steps_done++;
                    r->newton_its += f.newton_its;
                    r->gmres_its += f.gmres_its;
                    r->retries += f.retries;
                    r->t = f.t;
                    r->energy = f.energy;
                    r->mass = f.mass;
                    retire = r->steps_done >= r->steps;
                }
                if (retire) {
                    r->u.assign((size_t)r->grid.dim * r->c.size(), 0.0);
                    if (r->status == NKS_OK) nks_batch_get_fields(B, s, r->c.data(), r->eta.data(), r->u.data());
                    nks_batch_unload(B, s);
                    retiring.push_back(s);
                }
            }
        }
        std::lock_guard<std::mutex> lk(S->mu);
        for (auto &r : failed) {
            finish(S, r);
            G->occupied--;
        }
        for (int s : retiring) {
            finish(S, slot[s]);
            slot[s].reset();
            G->occupied--;
        }
        admit_locked(S);
        S->cv.notify_all();
    }
    if (B) nks_destroy(B);
    cudaStreamSynchronize(stream);
    cudaStreamDestroy(stream);
    std::lock_guard<std::mutex> lk(S->mu);
    S->used -= G->bytes;
    admit_locked(S);
    S->cv.notify_all();
}

}  // namespace

extern "C" {

void nks_server_default_opts(nks_server_opts *o)
{
    memset(o, 0, sizeof(*o));
    nks_default_opts(&o->opts);
    o->opts.precision = NKS_MIXED;
    o->opts.dt_mode = NKS_DT_ENERGY;
    o->mem_budget = 0;
    o->max_slots = 16;
    o->max_groups = 8;
    o->box_side_2d = 32;
    o->box_side_3d = 16;
}

int nks_server_create(const nks_coeffs *coeffs, const nks_server_opts *opts, nks_server **out)
{
    if (!coeffs || !opts || !out || opts->max_slots < 1 || opts->max_groups < 1 || opts->box_side_2d < 4 ||
        opts->box_side_3d < 4) {
        set_thread_error("nks_server_create: invalid argument");
        return NKS_EINVAL;
    }
    nks_server *S = new nks_server();
    S->coeffs = *coeffs;
    S->so = *opts;
    cudaGetDevice(&S->device);
    if (S->so.mem_budget == 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        S->so.mem_budget = (size_t)(0.8 * (double)fr);
    }
    S->t0 = Clock::now();
    *out = S;
    return NKS_OK;
}

int nks_server_submit(nks_server *S, const nks_grid *grid, const double *c, const double *eta, int steps,
                      long long *id)
{
    if (!S || !grid || !c || !eta || steps < 1 || grid->dim < 1 || grid->dim > 3) {
        set_thread_error("nks_server_submit: invalid argument");
        return NKS_EINVAL;
    }
    auto r = std::make_shared<Request>();
    r->grid = *grid;
    for (int J = grid->dim; J < 3; J++) r->grid.n[J] = 1;
    long long N = 1;
    for (int J = 0; J < grid->dim; J++) N *= grid->n[J];
    const long long ne = S->coeffs.n_eta == 3 ? 3 : 1;  // order-parameter planes
    r->c.assign(c, c + N);
    r->eta.assign(eta, eta + ne * N);
    r->steps = steps;
    const ShapeKey k = key_of(r->grid);
    bool need = false;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        need = S->slot_bytes.find(k) == S->slot_bytes.end();
    }
    if (need) {
        const size_t b = measure_slot(S, r->grid);
        if (b == 0) {
            set_thread_error("nks_server_submit: this grid cannot be set up (decomposition or memory)");
            return NKS_EINVAL;
        }
        std::lock_guard<std::mutex> lk(S->mu);
        S->slot_bytes[k] = b;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->slot_bytes[k] > S->so.mem_budget) {
        set_thread_error("nks_server_submit: one slot of this grid exceeds the memory budget");
        return NKS_ENOMEM;
    }
    r->id = S->next_id++;
    r->t_submit = S->now();
    S->all[r->id] = r;
    S->waiting.push_back(r);
    admit_locked(S);
    if (id) *id = r->id;
    return NKS_OK;
}

// wait for request id (timeout_s < 0: no limit); copies its result and final
// fields (c: N, eta: n_eta N, u: d N doubles; any may be NULL) and forgets it
int nks_server_wait(nks_server *S, long long id, nks_request_result *res, double *c, double *eta, double *u,
                    double timeout_s)
{
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) {
        set_thread_error("nks_server_wait: unknown request id");
        return NKS_EINVAL;
    }
    std::shared_ptr<Request> r = it->second;
    auto ready = [&] { return r->done; };
    if (timeout_s < 0.0) S->cv.wait(lk, ready);
    else if (!S->cv.wait_for(lk, std::chrono::duration<double>(timeout_s), ready)) return NKS_ETIMEOUT;
    if (res) {
        res->id = r->id;
        res->status = r->status;
        res->steps = r->steps_done;
        res->newton_its = r->newton_its;
        res->gmres_its = r->gmres_its;
        res->retries = r->retries;
        res->t_submit = r->t_submit;
        res->t_admit = r->t_admit;
        res->t_done = r->t_done;
        res->t = r->t;
        res->energy = r->energy;
        res->mass = r->mass;
        res->points = (long long)r->c.size();
    }
    const size_t N = r->c.size();
    if (r->status == NKS_OK) {
        if (c) memcpy(c, r->c.data(), N * sizeof(double));
        if (eta) memcpy(eta, r->eta.data(), r->eta.size() * sizeof(double));
        if (u && !r->u.empty()) memcpy(u, r->u.data(), r->u.size() * sizeof(double));
    }
    S->all.erase(it);
    return NKS_OK;
}

int nks_server_status(nks_server *S, nks_server_state *st)
{
    std::lock_guard<std::mutex> lk(S->mu);
    st->waiting = (int)S->waiting.size();
    st->groups = (int)S->groups.size();
    int inflight = 0;
    for (auto &g : S->groups) inflight += g.second->occupied;
    st->in_flight = inflight;
    st->bytes_reserved = S->used;
    st->mem_budget = S->so.mem_budget;
    return NKS_OK;
}

void nks_server_destroy(nks_server *S)
{
    if (!S) return;
    // wait for every submitted request, then for the workers
    {
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv.wait(lk, [&] {
            for (auto &kv : S->all)
                if (!kv.second->done) return false;
            return S->waiting.empty() && S->groups.empty();
        });
    }
    for (auto &g : S->retired)
        if (g->worker.joinable()) g->worker.join();
    delete S;
}

}  // extern "C"
