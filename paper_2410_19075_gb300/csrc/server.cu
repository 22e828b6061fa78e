// Serving: a native request loop with continuous batching.
//
// Device memory: the budget is one arena allocated once; jobs get first-fit
// blocks of it, so admission and retirement never call cudaMalloc or cudaFree.
//
// Jobs (one network each: model, topology, size, parameters, initial state,
// horizon) arrive through srv_submit at any time.  A worker thread admits them
// in arrival order while the resident jobs' device memory stays within the HBM
// budget and a slot is free, keeps their state on the device, advances every
// resident job together through the batched stage kernels (one launch per RK4
// stage for all ring jobs of a model; lattice jobs by their own kernels) in chunks
// of chunk_steps, and retires a job as soon as its horizon is reached: its step
// budget stops it exactly inside a chunk, its final state and order parameters
// are copied to host memory and its device memory is released, which lets the
// next queued jobs in.  The batch is re-formed whenever membership changes.
// Each result is bit-for-bit the same as the job run alone, because every
// window sum is exact and each job keeps its own buffers.
//
// With max_slots = 1 the loop runs one job at a time on the plain path
// (sim_step), which is the baseline the batched service is compared with.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"
#include "sim.h"

namespace {

double now_s()
{
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over one device arena (the HBM budget), so that admitting
// and retiring jobs never calls cudaMalloc/cudaFree (which synchronise the device).
class Arena {
  public:
    bool init(size_t bytes)
    {
        if (base_) return true;
        if (cudaMalloc(&base_, bytes) != cudaSuccess) {
            cudaGetLastError();
            base_ = nullptr;
            return false;
        }
        free_[0] = bytes;
        return true;
    }
    void release_all()
    {
        if (base_) cudaFree(base_);
        base_ = nullptr;
        free_.clear();
    }
    // offset of a free block of `bytes` (multiple of 256), or -1
    int64_t take(size_t bytes)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t at = it->first, rest = it->second - bytes;
                free_.erase(it);
                if (rest) free_[at + bytes] = rest;
                return (int64_t)at;
            }
        }
        return -1;
    }
    void give(size_t at, size_t bytes)
    {
        auto it = free_.emplace(at, bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    char *base() const { return static_cast<char *>(base_); }

  private:
    void *base_ = nullptr;
    std::map<size_t, size_t> free_; // offset -> size
};

struct Job {
    int64_t id = 0;
    bool waited_hbm = false; // its admission was held back by the budget or by fragmentation
    int64_t arena_at = -1;
    int model = 0, topo = 0;
    int64_t N = 0, R = 0, steps = 0, left = 0;
    double dt = 0.0;
    std::vector<double> params, init, npar;
    size_t bytes = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    sim_t h = nullptr;
    bool done = false;
    int status = SIM_OK;
    std::vector<double> result, order;
};

} // namespace

struct srv_handle {
    size_t budget = 0;
    int device = 0;
    int max_slots = 1;
    int64_t chunk = 64;
    cudaStream_t stream = nullptr;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Job *> queue;
    std::vector<Job *> resident; // touched by the worker only
    std::map<int64_t, Job *> jobs;
    std::thread worker;
    bool stop = false;
    int64_t next_id = 0;
    size_t used = 0;
    size_t peak_used = 0;     // largest `used` seen at any admission
    int64_t hbm_waits = 0;    // jobs whose admission waited for device memory while a slot was free
    // statistics
    int64_t completed = 0, node_steps = 0, batches_formed = 0, ticks = 0;
    // worker time by phase (seconds): admission, batch formation, stepping
    // (launches and the wait for the chunk), retirement, waiting for work
    double t_phase[5] = {0, 0, 0, 0, 0};
    // batch state (worker only)
    std::map<double, sim_batch_t> batches;
    bool membership_changed = true;
    Arena arena;
};

namespace {

int64_t nodes_of(const Job &j)
{
    return j.topo == SIM_RING ? j.N : j.topo == SIM_DISK2D ? j.N * j.N : j.N * j.N * j.N;
}
int dim_of(int model) { return model == SIM_KS ? 1 : model == SIM_HH ? 4 : 2; }

void destroy_batches(srv_t s)
{
    for (auto &kv : s->batches) sim_batch_destroy(kv.second);
    s->batches.clear();
}

// Create the job's network in its arena block (outside the lock).
void admit(srv_t s, Job *j)
{
    j->t_admit = now_s();
    sim_t h = nullptr;
    int st = sim_create_in(&h, j->model, j->topo, j->N, j->R, j->params.data(), (int)j->params.size(), 0,
                           s->arena.base() + j->arena_at, j->bytes, s->stream);
    if (st == SIM_OK && j->model == SIM_HH && !j->npar.empty())
        st = sim_set_node_param(h, 0, j->npar.data(), (int64_t)j->npar.size());
    if (st == SIM_OK) st = sim_set_state(h, j->init.data(), (int64_t)j->init.size());
    if (st != SIM_OK) {
        if (h) sim_destroy(h);
        j->status = st;
        j->h = nullptr;
        return;
    }
    j->h = h;
    j->left = j->steps;
    j->init.clear();
    j->init.shrink_to_fit();
}

void retire(srv_t s, Job *j)
{
    j->result.resize((size_t)dim_of(j->model) * nodes_of(*j));
    int st = sim_get_state(j->h, j->result.data(), (int64_t)j->result.size());
    if (st == SIM_OK && (j->model == SIM_KS || j->model == SIM_KSI)) {
        j->order.resize((size_t)j->steps + 1);
        int64_t n = 0;
        st = sim_observables(j->h, j->order.data(), (int64_t)j->order.size(), &n);
        j->order.resize((size_t)n);
    }
    j->status = st;
    sim_destroy(j->h);
    j->h = nullptr;
    j->t_done = now_s();
}

void worker_loop(srv_t s)
{
    cudaSetDevice(s->device);
    for (;;) {
        // 1. admission: FIFO while a slot is free and the budget allows
        std::vector<Job *> to_admit;
        double t0 = now_s();
        {
            std::unique_lock<std::mutex> lock(s->mu);
            if (s->stop) break;
            if (s->resident.empty() && s->queue.empty()) {
                s->cv_work.wait(lock, [&] { return s->stop || !s->queue.empty(); });
                const double t = now_s();
                s->t_phase[4] += t - t0;
                t0 = t;
            }
            if (s->stop) break;
            if (!s->queue.empty() && !s->arena.init(s->budget)) {
                // the budget itself cannot be allocated: fail every queued job
                while (!s->queue.empty()) {
                    Job *j = s->queue.front();
                    s->queue.pop_front();
                    j->status = SIM_ENOMEM;
                    j->done = true;
                }
                s->cv_done.notify_all();
                continue;
            }
            while (!s->queue.empty() && (int)(s->resident.size() + to_admit.size()) < s->max_slots) {
                Job *j = s->queue.front();
                const int64_t at = s->used + j->bytes > s->budget ? -1 : s->arena.take(j->bytes);
                if (at < 0) { // over the budget, or fragmented: wait for retirements
                    if (!j->waited_hbm) {
                        j->waited_hbm = true;
                        s->hbm_waits++;
                    }
                    break;
                }
                j->arena_at = at;
                s->queue.pop_front();
                s->used += j->bytes;
                if (s->used > s->peak_used) s->peak_used = s->used;
                to_admit.push_back(j);
            }
        }
        for (Job *j : to_admit) {
            admit(s, j);

            if (j->h) {
                s->resident.push_back(j);
                s->membership_changed = true;
            } else {
                std::lock_guard<std::mutex> lock(s->mu);
                s->used -= j->bytes;
                s->arena.give((size_t)j->arena_at, j->bytes);
                j->done = true;
                j->t_done = now_s();
                s->cv_done.notify_all();
            }
        }
        double t1 = now_s();
        s->t_phase[0] += t1 - t0;
        if (s->resident.empty()) continue;

        // 2. advance the resident jobs by one chunk
        if (s->max_slots == 1) {
            // plain path: one job at a time
            Job *j = s->resident[0];
            const int64_t n = j->left < s->chunk ? j->left : s->chunk;
            int st = sim_step(j->h, n, j->dt);
            if (st == SIM_OK) st = sim_sync(j->h);
            if (st != SIM_OK) j->status = st;
            j->left -= n;
            s->node_steps += n * nodes_of(*j);
        } else {
            if (s->membership_changed) {
                destroy_batches(s);
                std::map<double, std::vector<Job *>> by_dt;
                for (Job *j : s->resident) by_dt[j->dt].push_back(j);
                for (auto &kv : by_dt) {
                    std::vector<sim_t> hs;
                    std::vector<int64_t> bud;
                    for (Job *j : kv.second) {
                        hs.push_back(j->h);
                        bud.push_back(j->topo == SIM_RING ? j->left : -1);
                    }
                    sim_batch_t b = nullptr;
                    int st = sim_batch_create(&b, hs.data(), (int)hs.size(), s->stream);
                    if (st == SIM_OK) st = sim_batch_set_budgets(b, bud.data());
                    if (st != SIM_OK) {
                        for (Job *j : kv.second) j->status = st;
                        if (b) sim_batch_destroy(b);
                        continue;
                    }
                    s->batches[kv.first] = b;
                }
                s->membership_changed = false;
                s->batches_formed++;
                const double t = now_s();
                s->t_phase[1] += t - t1;
                t1 = t;
            }
            // lattice jobs carry no device budget: step the chunk only as far as
            // the shortest lattice horizon
            int64_t n = s->chunk;
            for (Job *j : s->resident)
                if (j->topo != SIM_RING && j->left < n) n = j->left;
            for (auto &kv : s->batches) {
                int st = sim_batch_step(kv.second, n, kv.first);
                if (st == SIM_OK) st = sim_batch_sync(kv.second);
                if (st != SIM_OK)
                    for (Job *j : s->resident)
                        if (j->dt == kv.first) j->status = st;
            }
            for (Job *j : s->resident) {
                const int64_t d = j->left < n ? j->left : n;
                j->left -= d;
                s->node_steps += d * nodes_of(*j);
            }
        }
        s->ticks++;
        const double t2 = now_s();
        s->t_phase[2] += t2 - t1;

        // 3. retire finished jobs
        std::vector<Job *> still;
        std::vector<Job *> finished;
        for (Job *j : s->resident) {
            if (j->left <= 0 || j->status != SIM_OK) finished.push_back(j);
            else still.push_back(j);
        }
        if (!finished.empty()) {
            for (Job *j : finished) {
                const int keep = j->status;
                retire(s, j);
                if (keep != SIM_OK) j->status = keep;
            }
            s->resident.swap(still);
            s->membership_changed = true;
            if (s->max_slots > 1) destroy_batches(s);
            std::lock_guard<std::mutex> lock(s->mu);
            for (Job *j : finished) {
                s->used -= j->bytes;
                s->arena.give((size_t)j->arena_at, j->bytes);
                j->done = true;
                s->completed++;
            }
            s->cv_done.notify_all();
        }
        s->t_phase[3] += now_s() - t2;
    }
    destroy_batches(s);
    for (Job *j : s->resident)
        if (j->h) sim_destroy(j->h);
    s->resident.clear();
    cudaStreamSynchronize(s->stream);
    s->arena.release_all();
}

} // namespace

extern "C" {

int srv_create(srv_t *out, size_t hbm_budget_bytes, int max_slots, int64_t chunk_steps, void *stream)
{
    if (!out || max_slots < 1 || chunk_steps < 1 || hbm_budget_bytes == 0) return SIM_EINVAL;
    srv_t s = new srv_handle();
    s->budget = hbm_budget_bytes;
    s->max_slots = max_slots;
    s->chunk = chunk_steps;
    s->stream = static_cast<cudaStream_t>(stream);
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return SIM_EDEVICE;
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return SIM_OK;
}

int srv_submit(srv_t s, int model, int topology, int64_t N, int64_t radius, const double *params, int n_params,
               const double *host_init_state, const double *host_node_param, int64_t n_steps, double dt,
               int64_t *job_id)
{
    if (!s || !job_id || !host_init_state || n_steps < 1 || !(dt > 0.0)) return SIM_EINVAL;
    const size_t bytes = (sim_workspace_bytes(model, topology, N, radius) + 255) / 256 * 256;
    if (bytes == 0) return SIM_EINVAL;
    if (bytes > s->budget) return SIM_ENOMEM;
    Job *j = new Job();
    j->model = model;
    j->topo = topology;
    j->N = N;
    j->R = radius;
    j->steps = n_steps;
    j->dt = dt;
    j->params.assign(params, params + n_params);
    const int64_t n = dim_of(model) * (topology == SIM_RING ? N : topology == SIM_DISK2D ? N * N : N * N * N);
    j->init.assign(host_init_state, host_init_state + n);
    if (host_node_param && model == SIM_HH) j->npar.assign(host_node_param, host_node_param + N);
    j->bytes = bytes;
    j->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lock(s->mu);
        j->id = s->next_id++;
        s->jobs[j->id] = j;
        s->queue.push_back(j);
    }
    s->cv_work.notify_one();
    *job_id = j->id;
    return SIM_OK;
}

int srv_poll(srv_t s, int64_t job_id, int *done, double *host_state_out, int64_t n_values, double *host_order_out,
             int64_t max_order, int64_t *n_order, double *times_out)
{
    if (!s || !done) return SIM_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return SIM_EINVAL;
    Job *j = it->second;
    *done = j->done ? 1 : 0;
    if (!j->done) return SIM_OK;
    const int st = j->status;
    if (host_state_out) {
        if (n_values != (int64_t)j->result.size()) return SIM_EINVAL;
        std::copy(j->result.begin(), j->result.end(), host_state_out);
    }
    if (n_order) {
        const int64_t n = (int64_t)j->order.size() < max_order ? (int64_t)j->order.size() : max_order;
        if (host_order_out) std::copy(j->order.begin(), j->order.begin() + n, host_order_out);
        *n_order = n;
    }
    if (times_out) {
        times_out[0] = j->t_submit;
        times_out[1] = j->t_admit;
        times_out[2] = j->t_done;
    }
    s->jobs.erase(it);
    delete j;
    return st;
}

int srv_wait_idle(srv_t s)
{
    if (!s) return SIM_EINVAL;
    std::unique_lock<std::mutex> lock(s->mu);
    s->cv_done.wait(lock, [&] {
        if (!s->queue.empty()) return false;
        for (auto &kv : s->jobs)
            if (!kv.second->done) return false;
        return true;
    });
    return SIM_OK;
}

int srv_timings(srv_t s, double *out5)
{
    if (!s || !out5) return SIM_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    for (int k = 0; k < 5; ++k) out5[k] = s->t_phase[k];
    return SIM_OK;
}

int srv_stats(srv_t s, int64_t *out6)
{
    if (!s || !out6) return SIM_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    int64_t pending = 0;
    for (auto &kv : s->jobs)
        if (!kv.second->done) ++pending;
    out6[0] = s->completed;
    out6[1] = pending;
    out6[2] = (int64_t)s->queue.size();
    out6[3] = s->node_steps;
    out6[4] = s->batches_formed;
    out6[5] = (int64_t)s->used;
    return SIM_OK;
}

int srv_memory(srv_t s, int64_t *out3)
{
    if (!s || !out3) return SIM_EINVAL;
    std::lock_guard<std::mutex> lock(s->mu);
    out3[0] = (int64_t)s->used;
    out3[1] = (int64_t)s->peak_used;
    out3[2] = s->hbm_waits;
    return SIM_OK;
}

void srv_destroy(srv_t s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto &kv : s->jobs) delete kv.second;
    delete s;
}

} // extern "C"
