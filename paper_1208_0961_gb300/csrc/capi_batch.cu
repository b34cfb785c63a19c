// Batch C ABI (include/cuba.h): many independent simulations in one arena.
//
// Residents occupy consecutive particle ranges and consecutive global cell
// ranges in admission order (the kernels locate a particle's or a cell's
// simulation by binary search over these offsets).  Admission appends; a
// retirement compacts the arena by copying the survivors into the other
// state buffer.  The descriptor table lives on the device, where the step
// counters advance; the host re-reads it before changing the table.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/cuba.h"
#include "engine.cuh"
#include "host.h"

using namespace cuba;
using namespace cuba::host;

namespace {

struct Member {
    int32_t id;
    cuba_params params;
    SimDesc desc;  // host copy (step counter refreshed from the device)
};

}  // namespace

struct cuba_batch {
    cuba_batch_config cfg;
    Arena A;
    StepGraphs graphs;
    std::vector<Member> members;      // arena order
    std::vector<uint32_t> free_slots; // counter rows not in use
    int32_t next_id = 1;
    double* d_obs = nullptr;          // observables scratch (max_cells x 20 bytes)
    double* d_tot = nullptr;
};

namespace {

int find_member(const cuba_batch* b, int32_t id)
{
    for (size_t k = 0; k < b->members.size(); ++k)
        if (b->members[k].id == id) return (int)k;
    return -1;
}

// Refresh the host copies of the descriptors from the device (step counters,
// simulated time, the adaptive step's constants).
int pull_table(cuba_batch* b)
{
    const size_t n = b->members.size();
    if (!n) return CUBA_OK;
    std::vector<SimDesc> t(n);
    CUDA_TRY(cudaDeviceSynchronize(), "sync");
    CUDA_TRY(cudaMemcpy(t.data(), b->A.d_sims, n * sizeof(SimDesc), cudaMemcpyDeviceToHost), "read table");
    // the device advances the step counter, the simulated time and (adaptive
    // dt) the step's constants; the layout fields agree with the host's
    for (size_t k = 0; k < n; ++k) b->members[k].desc = t[k];
    return CUBA_OK;
}

// Recompute offsets from the member order and upload the table.
int push_table(cuba_batch* b)
{
    Arena& A = b->A;
    uint32_t p = 0, c = 0;
    std::vector<SimDesc> t;
    t.reserve(b->members.size());
    for (Member& m : b->members) {
        m.desc.p_off = p;
        m.desc.cell_off = c;
        p += m.desc.np;
        c += m.desc.ncells;
        t.push_back(m.desc);
    }
    A.np = p;
    A.ncells = c;
    A.nsims = (int)b->members.size();
    if (!t.empty())
        CUDA_TRY(cudaMemcpy(A.d_sims, t.data(), t.size() * sizeof(SimDesc), cudaMemcpyHostToDevice), "upload table");
    set_key_param(A, t.data(), (int)t.size());
    return CUBA_OK;
}

int admit(cuba_batch* b, const cuba_params* params, int64_t n, int32_t* id, SimDesc* out_desc, int* index)
{
    if (!b || !params || !id) return fail(CUBA_ERR_INVALID, "bad arguments");
    SimDesc S;
    int rc = make_desc(params, &S);
    if (rc) return rc;
    if (params->precision != b->cfg.precision) return fail(CUBA_ERR_INVALID, "precision differs from the batch's");
    if (n < 0) return fail(CUBA_ERR_INVALID, "n must be >= 0");
    const Arena& A = b->A;
    if ((int)b->members.size() >= b->cfg.max_sims || b->free_slots.empty())
        return fail(CUBA_ERR_CAPACITY, "batch holds %d simulations already", (int)b->members.size());
    if ((uint64_t)A.np + (uint64_t)n > A.pcap)
        return fail(CUBA_ERR_CAPACITY, "no room for %lld particles (%u of %u in use)", (long long)n, A.np, A.pcap);
    if ((uint64_t)A.ncells + S.ncells > A.ccap)
        return fail(CUBA_ERR_CAPACITY, "no room for %u cells (%u of %u in use)", S.ncells, A.ncells, A.ccap);
    rc = pull_table(b);
    if (rc) return rc;
    S.np = (uint32_t)n;
    S.step = 0;
    S.stat_slot = b->free_slots.back();
    Member m;
    m.id = b->next_id++;
    m.params = *params;
    m.desc = S;
    b->members.push_back(m);
    b->free_slots.pop_back();
    CUDA_TRY(cudaMemset(b->A.stats + (size_t)S.stat_slot * kStatCount, 0, kStatCount * 8), "clear counters");
    rc = push_table(b);
    if (rc) return rc;
    *id = m.id;
    *index = (int)b->members.size() - 1;
    *out_desc = b->members.back().desc;
    return CUBA_OK;
}

// Undo an admission whose state could not be produced.
void unadmit(cuba_batch* b)
{
    b->free_slots.push_back(b->members.back().desc.stat_slot);
    b->members.pop_back();
    push_table(b);
}

// Sort the newly admitted (last) member's particles and size the lists.
int settle(cuba_batch* b, cudaStream_t st)
{
    const int k = (int)b->members.size() - 1;
    int rc = settle_arena(b->A, st, nullptr, k, &b->members[k].desc);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(st), "sync");
    return CUBA_OK;
}

}  // namespace

extern "C" {

int64_t cuba_batch_bytes(const cuba_batch_config* cfg)
{
    if (!cfg) return -1;
    if (cfg->precision != CUBA_FP32 && cfg->precision != CUBA_FP64) return -1;
    if (cfg->max_sims < 1 || cfg->max_sims > 65536) return -1;
    if (cfg->max_particles < 1 || cfg->max_particles > (int64_t)0x7FFFFFF0) return -1;
    if (cfg->max_cells < 1 || cfg->max_cells > (int64_t)(1 << 30)) return -1;
    return (int64_t)object_bytes(cfg->precision, (uint32_t)cfg->max_particles, (uint32_t)cfg->max_cells,
                                 cfg->max_sims);
}

static int create_batch(const cuba_batch_config* cfg, const cuba_allocator* mem, cuba_batch** out)
{
    if (!cfg || !out) return fail(CUBA_ERR_INVALID, "bad arguments");
    *out = nullptr;
    if (cfg->precision != CUBA_FP32 && cfg->precision != CUBA_FP64) return fail(CUBA_ERR_INVALID, "bad precision");
    if (cfg->max_sims < 1 || cfg->max_sims > 65536) return fail(CUBA_ERR_INVALID, "max_sims out of range");
    if (cfg->max_particles < 1 || cfg->max_particles > (int64_t)0x7FFFFFF0)
        return fail(CUBA_ERR_INVALID, "max_particles out of range");
    if (cfg->max_cells < 1 || cfg->max_cells > (int64_t)(1 << 30)) return fail(CUBA_ERR_INVALID, "max_cells out of range");
    if (kernels_init()) return fail(CUBA_ERR_CUDA, "kernel attribute setup failed");
    cuba_batch* b = new cuba_batch();
    b->cfg = *cfg;
    int rc = arena_alloc(b->A, cfg->precision, (uint32_t)cfg->max_particles, (uint32_t)cfg->max_cells, cfg->max_sims,
                         mem);
    if (!rc) rc = arena_dalloc(b->A, &b->d_obs, obs_scratch_bytes((uint32_t)cfg->max_cells), "observables");
    if (!rc) rc = arena_dalloc(b->A, &b->d_tot, kTotScratchBytes, "totals");
    if (rc) {
        cuba_batch_destroy(b);
        return rc;
    }
    for (int k = cfg->max_sims - 1; k >= 0; --k) b->free_slots.push_back((uint32_t)k);
    b->A.nsims = 0;
    b->A.np = 0;
    b->A.ncells = 0;
    *out = b;
    return CUBA_OK;
}

int cuba_batch_create(const cuba_batch_config* cfg, cuba_batch** out) { return create_batch(cfg, nullptr, out); }

int cuba_batch_create_with_allocator(const cuba_batch_config* cfg, const cuba_allocator* allocator, cuba_batch** out)
{
    if (!allocator || !allocator->alloc || !allocator->free)
        return fail(CUBA_ERR_INVALID, "allocator needs both alloc and free");
    return create_batch(cfg, allocator, out);
}

void cuba_batch_destroy(cuba_batch* b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    b->graphs.drop();
    arena_free(b->A);
    delete b;
}

int cuba_batch_add(cuba_batch* b, const cuba_params* params, int64_t n, const cuba_region* regions, int n_regions,
                   int32_t* id, void* stream)
{
    SimDesc S;
    int index = -1;
    int rc = admit(b, params, n, id, &S, &index);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    rc = sample_regions(b->A, index, S, n, regions, n_regions, params->L, st);
    if (rc) {
        unadmit(b);
        return rc;
    }
    return settle(b, st);
}

int cuba_batch_add_state(cuba_batch* b, const cuba_params* params, const void* soa, int64_t n, int32_t* id,
                         void* stream)
{
    if (n > 0 && !soa) return fail(CUBA_ERR_INVALID, "state is NULL");
    SimDesc S;
    int index = -1;
    int rc = admit(b, params, n, id, &S, &index);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    Arena& A = b->A;
    const size_t es = A.precision == CUBA_FP64 ? 8 : 4;
    for (int c = 0; c < 6; ++c) {
        cudaError_t e = cudaMemcpyAsync((char*)A.st[A.cur] + ((size_t)c * A.pcap + S.p_off) * es,
                                        (const char*)soa + (size_t)c * n * es, (size_t)n * es, cudaMemcpyDefault, st);
        if (e != cudaSuccess) {
            unadmit(b);
            return cuda_fail(e, "copy state in");
        }
    }
    return settle(b, st);
}

int cuba_batch_remove(cuba_batch* b, int32_t id)
{
    if (!b) return fail(CUBA_ERR_INVALID, "batch is NULL");
    const int k = find_member(b, id);
    if (k < 0) return fail(CUBA_ERR_INVALID, "no member with id %d", id);
    int rc = pull_table(b);
    if (rc) return rc;
    Arena& A = b->A;
    const bool last = k == (int)b->members.size() - 1;
    const SimDesc gone = b->members[k].desc;
    const uint32_t ncells_old = A.ncells;
    if (!last) {
        // copy every survivor to its new offset in the other state buffer
        const size_t es = A.precision == CUBA_FP64 ? 8 : 4;
        const char* src = (const char*)A.st[A.cur];
        char* dst = (char*)A.st[A.cur ^ 1];
        uint32_t p_new = 0;
        for (size_t j = 0; j < b->members.size(); ++j) {
            if ((int)j == k) continue;
            const SimDesc& d = b->members[j].desc;
            for (int c = 0; c < 6; ++c)
                CUDA_TRY(cudaMemcpyAsync(dst + ((size_t)c * A.pcap + p_new) * es, src + ((size_t)c * A.pcap + d.p_off) * es,
                                         (size_t)d.np * es, cudaMemcpyDeviceToDevice, 0),
                         "compact");
            p_new += d.np;
        }
        A.cur ^= 1;
        // the later members keep their order: their cell_start entries move
        // down by the removed member's cells and drop its particle count
        // (through the per-cell work table as scratch, which the list sizing
        // below recomputes)
        const uint32_t from = gone.cell_off + gone.ncells;
        const size_t cnt = (size_t)ncells_old - from + 1;
        uint32_t* tmp = reinterpret_cast<uint32_t*>(A.cell_work);
        CUDA_TRY(cudaMemcpyAsync(tmp, A.cell_start + from, cnt * 4, cudaMemcpyDeviceToDevice, 0), "cell_start");
        CUDA_TRY(cudaMemcpyAsync(A.cell_start + gone.cell_off, tmp, cnt * 4, cudaMemcpyDeviceToDevice, 0),
                 "cell_start");
        if (launch_add_u32(A.cell_start + gone.cell_off, (uint32_t)cnt, 0u - gone.np, 0))
            return fail(CUBA_ERR_CUDA, "cell_start shift failed");
    }
    b->free_slots.push_back(b->members[k].desc.stat_slot);
    b->members.erase(b->members.begin() + k);
    rc = push_table(b);
    if (rc) return rc;
    if (A.np == 0) return CUBA_OK;
    rc = settle_arena(A, 0, nullptr, kSettleNoSort, nullptr);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(0), "sync");
    return CUBA_OK;
}

int cuba_batch_step(cuba_batch* b, int n_steps, void* stream)
{
    if (!b || n_steps < 0) return fail(CUBA_ERR_INVALID, "bad arguments");
    if (b->members.empty()) return CUBA_OK;
    return b->graphs.run(b->A, n_steps, (cudaStream_t)stream);
}

int cuba_batch_observables(cuba_batch* b, int32_t id, double* T00, double* T0x, int32_t* counts, void* stream)
{
    if (!b) return fail(CUBA_ERR_INVALID, "batch is NULL");
    const int k = find_member(b, id);
    if (k < 0) return fail(CUBA_ERR_INVALID, "no member with id %d", id);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nc = b->members[k].desc.ncells;
    double* dT00 = b->d_obs;
    double* dT0x = b->d_obs + nc;
    int32_t* dcnt = reinterpret_cast<int32_t*>(b->d_obs + 2 * nc);
    if (launch_observables(b->A, k, dT00, dT0x, dcnt, st)) return fail(CUBA_ERR_CUDA, "observables launch failed");
    if (T00) CUDA_TRY(cudaMemcpyAsync(T00, dT00, nc * 8, cudaMemcpyDefault, st), "copy T00");
    if (T0x) CUDA_TRY(cudaMemcpyAsync(T0x, dT0x, nc * 8, cudaMemcpyDefault, st), "copy T0x");
    if (counts) CUDA_TRY(cudaMemcpyAsync(counts, dcnt, nc * 4, cudaMemcpyDefault, st), "copy counts");
    CUDA_TRY(cudaStreamSynchronize(st), "sync");
    return read_kernel_errors(b->A);
}

int cuba_batch_totals(cuba_batch* b, int32_t id, double out[4], int64_t* n, void* stream)
{
    if (!b || !out) return fail(CUBA_ERR_INVALID, "bad arguments");
    const int k = find_member(b, id);
    if (k < 0) return fail(CUBA_ERR_INVALID, "no member with id %d", id);
    cudaStream_t st = (cudaStream_t)stream;
    if (launch_totals(b->A, k, b->d_tot, st)) return fail(CUBA_ERR_CUDA, "totals launch failed");
    CUDA_TRY(cudaMemcpyAsync(out, b->d_tot, 4 * sizeof(double), cudaMemcpyDefault, st), "copy totals");
    CUDA_TRY(cudaStreamSynchronize(st), "sync");
    if (n) *n = b->members[k].desc.np;
    return read_kernel_errors(b->A);
}

int cuba_batch_stats(cuba_batch* b, int32_t id, cuba_counters* out)
{
    if (!b || !out) return fail(CUBA_ERR_INVALID, "bad arguments");
    const int k = find_member(b, id);
    if (k < 0) return fail(CUBA_ERR_INVALID, "no member with id %d", id);
    unsigned long long h[kStatCount];
    CUDA_TRY(cudaDeviceSynchronize(), "sync");
    CUDA_TRY(cudaMemcpy(h, b->A.stats + (size_t)b->members[k].desc.stat_slot * kStatCount, sizeof(h),
                        cudaMemcpyDeviceToHost),
             "read stats");
    out->steps = (int64_t)h[kStatSteps];
    out->pair_tests = (int64_t)h[kStatPairTests];
    out->accepted = (int64_t)h[kStatAccepted];
    out->executed = (int64_t)h[kStatExecuted];
    out->reflections = (int64_t)h[kStatReflections];
    out->fp64_boosts = (int64_t)h[kStatFp64Boosts];
    out->overflow = (int64_t)h[kStatOverflow];
    out->candidates = (int64_t)h[kStatCandidates];
    return read_kernel_errors(b->A);
}

int cuba_batch_get_state(cuba_batch* b, int32_t id, void* out, void* stream)
{
    if (!b) return fail(CUBA_ERR_INVALID, "batch is NULL");
    const int k = find_member(b, id);
    if (k < 0) return fail(CUBA_ERR_INVALID, "no member with id %d", id);
    const SimDesc& d = b->members[k].desc;
    if (!out && d.np) return fail(CUBA_ERR_INVALID, "out is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const Arena& A = b->A;
    const size_t es = A.precision == CUBA_FP64 ? 8 : 4;
    CUDA_TRY(cudaDeviceSynchronize(), "sync");
    for (int c = 0; c < 6; ++c)
        CUDA_TRY(cudaMemcpyAsync((char*)out + (size_t)c * d.np * es,
                                 (const char*)A.st[A.cur] + ((size_t)c * A.pcap + d.p_off) * es, (size_t)d.np * es,
                                 cudaMemcpyDefault, st),
                 "copy state out");
    CUDA_TRY(cudaStreamSynchronize(st), "sync");
    return read_kernel_errors(b->A);
}

int cuba_batch_get_step(cuba_batch* b, int32_t id, uint32_t* step)
{
    if (!b || !step) return fail(CUBA_ERR_INVALID, "bad arguments");
    const int k = find_member(b, id);
    if (k < 0) return fail(CUBA_ERR_INVALID, "no member with id %d", id);
    int rc = pull_table(b);
    if (rc) return rc;
    *step = b->members[k].desc.step;
    return CUBA_OK;
}

int cuba_batch_get_time(cuba_batch* b, int32_t id, double* time, double* last_dt)
{
    if (!b) return fail(CUBA_ERR_INVALID, "bad arguments");
    const int k = find_member(b, id);
    if (k < 0) return fail(CUBA_ERR_INVALID, "no member with id %d", id);
    int rc = pull_table(b);
    if (rc) return rc;
    if (time) *time = b->members[k].desc.time;
    if (last_dt) *last_dt = b->members[k].desc.dt;
    return CUBA_OK;
}

int cuba_batch_autotune(cuba_batch* b, int n_steps, int32_t* chosen, double* ms_per_candidate, void* stream)
{
    if (!b) return fail(CUBA_ERR_INVALID, "batch is NULL");
    return autotune_arena(b->A, n_steps, (cudaStream_t)stream, chosen, ms_per_candidate);
}

int cuba_batch_set_small_max(cuba_batch* b, int32_t small_max)
{
    if (!b) return fail(CUBA_ERR_INVALID, "batch is NULL");
    CUDA_TRY(cudaDeviceSynchronize(), "sync");
    return set_small_max(b->A, small_max);
}

int cuba_batch_set_launch_shape(cuba_batch* b, const cuba_launch_shape* shape)
{
    if (!b) return fail(CUBA_ERR_INVALID, "batch is NULL");
    CUDA_TRY(cudaDeviceSynchronize(), "sync");
    return set_launch_shape(b->A, shape);
}

int cuba_batch_get_launch_shape(cuba_batch* b, cuba_launch_shape* shape)
{
    if (!b || !shape) return fail(CUBA_ERR_INVALID, "bad arguments");
    get_launch_shape(b->A, shape);
    return CUBA_OK;
}

int cuba_batch_autotune_shape(cuba_batch* b, int n_steps, cuba_launch_shape* chosen, double* ms_per_candidate,
                              void* stream)
{
    if (!b) return fail(CUBA_ERR_INVALID, "batch is NULL");
    return autotune_shape(b->A, n_steps, (cudaStream_t)stream, chosen, ms_per_candidate);
}

int cuba_batch_usage(const cuba_batch* b, int32_t* n_sims, int64_t* n_particles, int64_t* n_cells)
{
    if (!b) return fail(CUBA_ERR_INVALID, "batch is NULL");
    if (n_sims) *n_sims = (int32_t)b->members.size();
    if (n_particles) *n_particles = b->A.np;
    if (n_cells) *n_cells = b->A.ncells;
    return CUBA_OK;
}

}  // extern "C"
