// C ABI of the library (include/cuba.h): parameter checks, device memory of a
// simulation, the step sequence and its CUDA-graph replay, observables.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/cuba.h"
#include "engine.cuh"
#include "host.h"

using namespace cuba;

namespace cuba {
namespace host {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    return fail(CUBA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}


constexpr double kDefaultGammaFp64 = 8.0;

// Validate parameters (Sec. 2, Sec. 5) and build the device descriptor.
int make_desc(const cuba_params* p, SimDesc* S)
{
    if (!p) return fail(CUBA_ERR_INVALID, "params is NULL");
    std::memset(S, 0, sizeof(*S));
    uint64_t nc = 1;
    for (int a = 0; a < 3; ++a) {
        if (!(p->L[a] > 0.0) || !std::isfinite(p->L[a])) return fail(CUBA_ERR_INVALID, "L[%d] must be > 0", a);
        if (p->n_cells[a] < 1) return fail(CUBA_ERR_INVALID, "n_cells[%d] must be >= 1", a);
        nc *= (uint64_t)p->n_cells[a];
        S->L[a] = p->L[a];
        S->n[a] = p->n_cells[a];
        S->dx[a] = p->L[a] / (double)p->n_cells[a];
        S->Lf[a] = (float)p->L[a];
        S->dxf[a] = (float)S->dx[a];
        S->rdx[a] = 1.0 / S->dx[a];
        S->rdxf[a] = (float)(1.0 / (double)S->dxf[a]);
        if (!(p->dt < S->dx[a]))
            return fail(CUBA_ERR_INVALID, "dt = %g must be below the cell edge %g on axis %d", p->dt, S->dx[a], a);
    }
    if (nc > (1ull << 30)) return fail(CUBA_ERR_INVALID, "too many cells (%llu)", (unsigned long long)nc);
    if (!(p->dt > 0.0)) return fail(CUBA_ERR_INVALID, "dt must be > 0");
    if (!(p->sigma_fm2 >= 0.0) || !std::isfinite(p->sigma_fm2)) return fail(CUBA_ERR_INVALID, "sigma must be >= 0");
    if (!(p->n_test > 0.0) || !std::isfinite(p->n_test)) return fail(CUBA_ERR_INVALID, "n_test must be > 0");
    if (p->precision != CUBA_FP32 && p->precision != CUBA_FP64) return fail(CUBA_ERR_INVALID, "bad precision");
    S->ncells = (uint32_t)nc;
    if (p->acceptance != CUBA_ACCEPT_ALL_PAIRS && p->acceptance != CUBA_ACCEPT_SKIP)
        return fail(CUBA_ERR_INVALID, "acceptance must be CUBA_ACCEPT_ALL_PAIRS or CUBA_ACCEPT_SKIP");
    if (!(p->kappa >= 0.0) || p->kappa > 0.5) return fail(CUBA_ERR_INVALID, "kappa must lie in [0, 1/2]");
    if (!(p->mass >= 0.0) || !std::isfinite(p->mass)) return fail(CUBA_ERR_INVALID, "mass must be >= 0");
    if (!(p->mu >= 0.0) || !std::isfinite(p->mu)) return fail(CUBA_ERR_INVALID, "mu must be >= 0");
    S->mass = p->mass;
    S->m2 = p->mass * p->mass;
    S->m2f = (float)S->m2;
    S->mu = p->mu;
    S->skip = p->acceptance == CUBA_ACCEPT_SKIP ? 1u : 0u;
    S->V = (S->dx[0] * S->dx[1]) * S->dx[2];
    S->sigma = p->sigma_fm2;
    S->n_test = p->n_test;
    S->kappa = p->kappa;
    S->dt_max = p->dt;
    S->dt = p->dt;
    S->time = 0.0;
    S->norm = p->n_test * S->V;
    derive_step_constants(*S);
    if (2.0 * S->C > 1.0) return fail(CUBA_ERR_P22, "P22 can reach 2C = %g > 1", 2.0 * S->C);
    if (S->skip && S->C > 0.0 && !(2.0001 * S->C < 1.0))
        return fail(CUBA_ERR_P22, "skip-ahead needs 2.0001 C < 1 (C = %g)", S->C);
    S->key0 = (uint32_t)p->seed;
    S->key1 = (uint32_t)(p->seed >> 32);
    S->gamma_fp64 = (float)(p->gamma_fp64 > 0.0 ? p->gamma_fp64 : kDefaultGammaFp64);
    S->step = 0;
    return CUBA_OK;
}

int arena_dalloc_raw(Arena& A, void** ptr, size_t bytes, const char* what)
{
    *ptr = nullptr;
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (A.mem_alloc) {
        p = A.mem_alloc(bytes, A.mem_ctx);
        if (!p) return fail(CUBA_ERR_OOM, "caller allocator returned NULL for %s (%zu bytes)", what, bytes);
        if (reinterpret_cast<uintptr_t>(p) % 256 != 0) {
            A.mem_free(p, bytes, A.mem_ctx);
            return fail(CUBA_ERR_INVALID, "caller allocator returned %p for %s: not 256-byte aligned", p, what);
        }
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(CUBA_ERR_OOM, "cudaMalloc %s (%zu bytes): %s", what, bytes, cudaGetErrorString(e));
        }
    }
    A.mem_blocks.push_back({p, bytes});
    *ptr = p;
    return CUBA_OK;
}

// A block goes back only once no kernel can still use it: cudaFree waits for
// the device itself; before a caller's free the device is synchronized here.
static void give_back(const Arena& A, const Arena::Block& b)
{
    if (A.mem_free) A.mem_free(b.ptr, b.bytes, A.mem_ctx);
    else cudaFree(b.ptr);
}

void arena_dfree(Arena& A, void* ptr)
{
    if (!ptr) return;
    for (size_t k = 0; k < A.mem_blocks.size(); ++k)
        if (A.mem_blocks[k].ptr == ptr) {
            if (A.mem_free) cudaDeviceSynchronize();
            give_back(A, A.mem_blocks[k]);
            A.mem_blocks.erase(A.mem_blocks.begin() + k);
            return;
        }
}

void arena_free(Arena& A)
{
    if (A.mem_free && !A.mem_blocks.empty()) cudaDeviceSynchronize();
    for (const Arena::Block& b : A.mem_blocks) give_back(A, b);
    A = Arena();
}

size_t scan_tmp_needed(uint32_t pcap, uint32_t ccap)
{
    const size_t tiles = (pcap + kSortTile - 1) / kSortTile + 1;
    const size_t n1 = (kBinBins * tiles + kScanTile - 1) / kScanTile;
    const size_t n2 = ((size_t)ccap + 1 + kScanTile - 1) / kScanTile;
    size_t need = std::max(n1 * sizeof(uint32_t), n2 * sizeof(uint2));
    need = std::max(need, bin_scan_bytes());
    return std::max<size_t>(need, 256 * 4 * sizeof(double)) + 256;
}

ArenaPlan arena_plan(int precision, uint32_t pcap, uint32_t ccap, int simcap)
{
    ArenaPlan P;
    const size_t es = precision == CUBA_FP64 ? sizeof(double) : sizeof(float);
    const size_t pc = std::max<uint32_t>(pcap, 1);
    P.state = 6 * pc * es;
    P.keys = pc * 4;
    P.perm = pc * 4;
    P.cell_start = ((size_t)ccap + 1) * 4;
    P.cell_work = ((size_t)ccap + 1) * sizeof(uint2);
    P.skip_work = ((size_t)ccap + 1) * sizeof(uint32_t);
    P.acc_count = (size_t)ccap * 4;
    P.active = (size_t)ccap * 4;
    P.radix_hist_cap = (uint32_t)(2 * kBinBins * ((pc + kSortTile - 1) / kSortTile + 1));
    P.radix_hist = (size_t)P.radix_hist_cap * 4;
    P.scan_tmp = scan_tmp_needed(pcap, ccap);
    P.counters = 16 * 4;
    // survivors of the random-byte filters: about one pair in 2^16, or
    // 2.0001 C of them (larger batches spill to in-place evaluation)
    P.surv_cap = std::max<uint32_t>(1u << 21, (uint32_t)(pc / 2));
    P.surv = (size_t)P.surv_cap * sizeof(uint4);
    P.used_bits = (pc / 32 + 2) * 4;
    if (ccap > (uint32_t)kBinBins && (size_t)27 * ccap <= ((size_t)1 << 29)) {
        P.nbr_cap = ccap;
        P.nbr_rel = (size_t)27 * ccap * 4;
        P.nbr_cs = ((size_t)ccap + 1) * 4;
    }
    P.stats = (size_t)simcap * kStatCount * 8;
    P.sims = ((size_t)simcap + 1) * sizeof(SimDesc);  // + one scratch descriptor (settle_member)
    return P;
}

int arena_alloc(Arena& A, int precision, uint32_t pcap, uint32_t ccap, int simcap, const cuba_allocator* mem)
{
    if (mem && (!mem->alloc || !mem->free)) return fail(CUBA_ERR_INVALID, "allocator needs both alloc and free");
    A.mem_alloc = mem ? mem->alloc : nullptr;
    A.mem_free = mem ? mem->free : nullptr;
    A.mem_ctx = mem ? mem->ctx : nullptr;
    A.precision = precision;
    A.pcap = pcap;
    A.ccap = ccap;
    A.simcap = simcap;
    const ArenaPlan P = arena_plan(precision, pcap, ccap, simcap);
    int rc = CUBA_OK;
    rc |= arena_dalloc(A, &A.st[0], P.state, "state");
    if (!rc) rc = arena_dalloc(A, &A.st[1], P.state, "state");
    if (!rc) rc = arena_dalloc(A, &A.key[0], P.keys, "keys");
    if (!rc) rc = arena_dalloc(A, &A.key[1], P.keys, "keys");
    if (!rc) rc = arena_dalloc(A, &A.idx[0], P.perm, "perm");
    if (!rc) rc = arena_dalloc(A, &A.idx[1], P.perm, "perm");
    if (!rc) rc = arena_dalloc(A, &A.cell_start, P.cell_start, "cell_start");
    if (!rc) rc = arena_dalloc(A, &A.cell_work, P.cell_work, "cell_work");
    if (!rc) rc = arena_dalloc(A, &A.skip_work, P.skip_work, "skip_work");
    if (!rc) rc = arena_dalloc(A, &A.acc_count, P.acc_count, "acc_count");
    if (!rc) rc = arena_dalloc(A, &A.active, P.active, "active");
    A.radix_hist_cap = P.radix_hist_cap;
    if (!rc) rc = arena_dalloc(A, &A.radix_hist, P.radix_hist, "radix_hist");
    A.scan_tmp_bytes = P.scan_tmp;
    if (!rc) rc = arena_dalloc(A, &A.scan_tmp, P.scan_tmp, "scan_tmp");
    if (!rc) rc = arena_dalloc(A, &A.counters, P.counters, "counters");
    A.surv_cap = P.surv_cap;
    if (!rc) rc = arena_dalloc(A, &A.surv, P.surv, "survivors");
    if (!rc) rc = arena_dalloc(A, &A.used_bits, P.used_bits, "used_bits");
    if (!rc && P.nbr_cap) {
        A.nbr_cap = P.nbr_cap;
        rc = arena_dalloc(A, &A.nbr_rel, P.nbr_rel, "neighbour offsets");
        if (!rc) rc = arena_dalloc(A, &A.nbr_cs, P.nbr_cs, "neighbour cell_start");
    }
    if (!rc) rc = arena_dalloc(A, &A.stats, P.stats, "stats");
    if (!rc) rc = arena_dalloc(A, &A.d_sims, P.sims, "sims");
    if (rc) {
        arena_free(A);
        return rc;
    }
    const size_t pc = std::max<uint32_t>(pcap, 1);
    cudaMemset(A.counters, 0, 16 * 4);
    cudaMemset(A.used_bits, 0, (pc / 32 + 2) * 4);
    cudaMemset(A.stats, 0, (size_t)simcap * kStatCount * 8);
    cudaMemset(A.cell_start, 0, ((size_t)ccap + 1) * 4);
    return CUBA_OK;
}

// Enqueue one step A1-A7 on every simulation of the arena (direct launch or
// capture).
int enqueue_step(Arena& A, cudaStream_t st)
{
    if (A.any_adapt && launch_adapt_dt(A, st)) return fail(CUBA_ERR_CUDA, "adaptive dt launch failed");
    if ((nbr_path(A) ? launch_step_nbr(A, st, nullptr) : launch_step_bin(A, st, nullptr)))
        return fail(CUBA_ERR_CUDA, "stream/sort launch failed");
    if (launch_cell_prep(A, st)) return fail(CUBA_ERR_CUDA, "cell preparation launch failed");
    if (launch_pair_tile(A, st)) return fail(CUBA_ERR_CUDA, "pair tile launch failed");
    if (launch_resolve(A, st)) return fail(CUBA_ERR_CUDA, "resolve launch failed");
    if (launch_advance(A, st)) return fail(CUBA_ERR_CUDA, "advance launch failed");
    return CUBA_OK;
}

// Largest-remainder split of n over weights T^3 V (ties to the lower index).
int split_counts(int64_t n, const cuba_region* R, int nreg, std::vector<int64_t>& counts)
{
    std::vector<double> w(nreg), frac(nreg);
    double wsum = 0.0;
    for (int r = 0; r < nreg; ++r) {
        double v = 1.0;
        for (int a = 0; a < 3; ++a) v *= (R[r].hi[a] - R[r].lo[a]);
        if (!(v > 0.0) || !(R[r].T > 0.0)) return fail(CUBA_ERR_INVALID, "region %d: empty box or T <= 0", r);
        w[r] = R[r].T * R[r].T * R[r].T * v;
        wsum += w[r];
    }
    counts.assign(nreg, 0);
    int64_t assigned = 0;
    for (int r = 0; r < nreg; ++r) {
        const double q = (double)n * w[r] / wsum;
        counts[r] = (int64_t)std::floor(q);
        frac[r] = q - (double)counts[r];
        assigned += counts[r];
    }
    while (assigned < n) {
        int best = 0;
        for (int r = 1; r < nreg; ++r)
            if (frac[r] > frac[best]) best = r;
        counts[best] += 1;
        frac[best] = -1.0;
        ++assigned;
    }
    return CUBA_OK;
}

// Sample thermal regions into particles [S.p_off, S.p_off + n) of the arena.
int sample_regions(Arena& A, int sim_index, const SimDesc& S, int64_t n, const cuba_region* regions, int n_regions,
                   const double* L, cudaStream_t st)
{
    if (!regions || n_regions < 1 || n_regions > 1024) return fail(CUBA_ERR_INVALID, "bad regions");
    for (int r = 0; r < n_regions; ++r)
        for (int a = 0; a < 3; ++a)
            if (!(regions[r].lo[a] >= 0.0) || !(regions[r].hi[a] <= L[a]) || !(regions[r].lo[a] < regions[r].hi[a]))
                return fail(CUBA_ERR_INVALID, "region %d is not a box inside [0, L]", r);
    std::vector<int64_t> counts;
    int rc = split_counts(n, regions, n_regions, counts);
    if (rc) return rc;
    std::vector<double> hreg(7 * n_regions);
    std::vector<uint64_t> first(n_regions);
    uint64_t acc = 0;
    for (int r = 0; r < n_regions; ++r) {
        for (int a = 0; a < 3; ++a) {
            hreg[7 * r + a] = regions[r].lo[a];
            hreg[7 * r + 3 + a] = regions[r].hi[a];
        }
        hreg[7 * r + 6] = regions[r].T;
        first[r] = acc;
        acc += (uint64_t)counts[r];
    }
    double* d_reg = nullptr;
    uint64_t* d_first = nullptr;
    if ((rc = arena_dalloc(A, &d_reg, hreg.size() * sizeof(double), "regions"))) return rc;
    if ((rc = arena_dalloc(A, &d_first, first.size() * sizeof(uint64_t), "regions"))) {
        arena_dfree(A, d_reg);
        return rc;
    }
    cudaMemcpy(d_reg, hreg.data(), hreg.size() * sizeof(double), cudaMemcpyHostToDevice);
    cudaMemcpy(d_first, first.data(), first.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
    cudaStreamSynchronize(st);
    if (launch_init_thermal(A, sim_index, S, d_reg, n_regions, d_first, st))
        rc = fail(CUBA_ERR_CUDA, "thermal sampling launch failed");
    cudaError_t e = cudaStreamSynchronize(st);
    arena_dfree(A, d_reg);
    arena_dfree(A, d_first);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "thermal sampling");
    return rc;
}

// The settling sort of one member's particles only (the others are sorted
// already and members own disjoint cell ranges, so the arena stays sorted):
// a view of the arena restricted to the member, with a descriptor copy at
// offset 0 in the scratch slot after the table, sorts into the other state
// buffer; the member's range is copied back and its cell_start entries
// shifted by its first particle.  desc: the member's descriptor.
static int settle_member(Arena& A, int member, const SimDesc& desc, cudaStream_t st)
{
    SimDesc L = desc;
    L.p_off = 0;
    L.cell_off = 0;
    SimDesc* scratch = A.d_sims + A.simcap;
    CUDA_TRY(cudaMemcpyAsync(scratch, &L, sizeof(SimDesc), cudaMemcpyHostToDevice, st), "member descriptor");
    const size_t es = A.precision == CUBA_FP64 ? 8 : 4;
    Arena V;  // borrows A's buffers; owns nothing
    V.precision = A.precision;
    V.pcap = A.pcap;
    V.ccap = A.ccap;
    V.np = desc.np;
    V.ncells = desc.ncells;
    V.nsims = 1;
    V.simcap = 1;
    V.st[0] = (char*)A.st[A.cur] + (size_t)desc.p_off * es;
    V.st[1] = (char*)A.st[A.cur ^ 1] + (size_t)desc.p_off * es;
    V.cur = 0;
    V.key[0] = A.key[0];
    V.key[1] = A.key[1];
    V.idx[0] = A.idx[0];
    V.idx[1] = A.idx[1];
    V.cell_start = A.cell_start + desc.cell_off;
    V.radix_hist = A.radix_hist;
    V.radix_hist_cap = A.radix_hist_cap;
    V.scan_tmp = A.scan_tmp;
    V.scan_tmp_bytes = A.scan_tmp_bytes;
    V.stats = A.stats;
    V.d_sims = scratch;
    (void)member;
    if (launch_settle_bin(V, st)) return fail(CUBA_ERR_CUDA, "sort launch failed");
    if (V.cur == 1)
        for (int c = 0; c < 6; ++c)
            CUDA_TRY(cudaMemcpyAsync((char*)V.st[0] + (size_t)c * A.pcap * es, (char*)V.st[1] + (size_t)c * A.pcap * es,
                                     (size_t)desc.np * es, cudaMemcpyDeviceToDevice, st),
                     "member state back");
    if (launch_add_u32(V.cell_start, desc.ncells + 1, desc.p_off, st))
        return fail(CUBA_ERR_CUDA, "cell_start shift failed");
    return CUBA_OK;
}

// Keys of the present positions, stable sort, and the size of the
// accepted-pair lists for the present occupancy (room for four times the
// present need plus 2^20 entries: occupancy changes as the system evolves).
// member >= 0: only that member's particles are sorted (desc: its
// descriptor); member == kSettleNoSort: the state and cell_start are sorted
// already.  Returns 1 in *realloc if the list buffer was replaced.
int settle_arena(Arena& A, cudaStream_t st, int* realloc, int member, const SimDesc* desc)
{
    if (realloc) *realloc = 0;
    if (member == kSettleNoSort) {
    } else if (member >= 0) {
        int rc = settle_member(A, member, *desc, st);
        if (rc) return rc;
    } else if (launch_settle_bin(A, st)) {
        return fail(CUBA_ERR_CUDA, "sort launch failed");
    }
    if (launch_cell_prep(A, st, 0)) return fail(CUBA_ERR_CUDA, "cell preparation failed");
    uint2 tot;
    CUDA_TRY(cudaMemcpyAsync(&tot, A.cell_work + A.ncells, sizeof(uint2), cudaMemcpyDeviceToHost, st), "read list size");
    CUDA_TRY(cudaStreamSynchronize(st), "sync");
    const uint64_t want = 4ull * tot.y + kMinAccEntries;
    if (want > A.acc_capacity) {
        if (A.acc) arena_dfree(A, A.acc);
        A.acc = nullptr;
        A.acc_capacity = 0;
        int rc = arena_dalloc(A, &A.acc, want * sizeof(unsigned long long), "accepted list");
        if (rc) return rc;
        A.acc_capacity = want;
        if (realloc) *realloc = 1;
    }
    return CUBA_OK;
}

int read_kernel_errors(Arena& A)
{
    uint32_t err = 0;
    CUDA_TRY(cudaDeviceSynchronize(), "synchronize");
    CUDA_TRY(cudaMemcpy(&err, A.counters + 1, 4, cudaMemcpyDeviceToHost), "read error flags");
    if (err) {
        cudaMemset(A.counters + 1, 0, 4);
        if (err & kErrMove)
            return fail(CUBA_ERR_INVALID, "a particle moved more than one cell along an axis in a step");
        if (err & kErrCapacity)
            return fail(CUBA_ERR_OVERFLOW, "accepted-pair lists of a step exceeded the allocated list; "
                                           "that step skipped its collisions");
        return fail(CUBA_ERR_OVERFLOW, "a cell's accepted-pair list overflowed; some accepted pairs were dropped");
    }
    return CUBA_OK;
}

void StepGraphs::drop()
{
    for (int k = 0; k < 2; ++k)
        if (g[k]) {
            cudaGraphExecDestroy(g[k]);
            g[k] = nullptr;
        }
}

// Launch n steps, capturing one graph per ping-pong buffer on first use; the
// graphs are dropped whenever the arena's layout changes.
int StepGraphs::run(Arena& A, int n, cudaStream_t st)
{
    if (np != A.np || acc != A.acc || trace != A.trace || nsims != A.nsims || ncells != A.ncells ||
        small_max != A.small_max || one_key != A.one_key || key0 != A.key_sched.k0[0] || key1 != A.key_sched.k1[0] ||
        modes != A.nbr_ok * 8 + A.any_adapt * 4 + A.any_skip * 2 + A.any_all_pairs || tile_nb != A.tile_nb ||
        small_nb != A.small_nb)
        drop();
    for (int k = 0; k < n; ++k) {
        const int which = A.cur;
        if (!g[which]) {
            if (!capture) CUDA_TRY(cudaStreamCreateWithFlags(&capture, cudaStreamNonBlocking), "capture stream");
            const int saved = A.cur;
            A.cur = which;
            cudaGraph_t graph = nullptr;
            CUDA_TRY(cudaStreamBeginCapture(capture, cudaStreamCaptureModeThreadLocal), "begin capture");
            int rc = enqueue_step(A, capture);
            cudaError_t e = cudaStreamEndCapture(capture, &graph);
            A.cur = saved;
            if (rc) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (e != cudaSuccess) return cuda_fail(e, "end capture");
            e = cudaGraphInstantiate(&g[which], graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "instantiate graph");
            np = A.np;
            acc = A.acc;
            trace = A.trace;
            nsims = A.nsims;
            ncells = A.ncells;
            small_max = A.small_max;
            one_key = A.one_key;
            key0 = A.key_sched.k0[0];
            key1 = A.key_sched.k1[0];
            modes = A.nbr_ok * 8 + A.any_adapt * 4 + A.any_skip * 2 + A.any_all_pairs;
            tile_nb = A.tile_nb;
            small_nb = A.small_nb;
        }
        CUDA_TRY(cudaGraphLaunch(g[which], st), "graph launch");
        A.cur ^= 1;
    }
    return CUBA_OK;
}

void set_key_param(Arena& A, const SimDesc* table, int n)
{
    A.one_key = n == 1;
    A.key_sched = n == 1 ? philox_schedule(table[0].key0, table[0].key1) : PhiloxKey{};
    A.any_skip = 0;
    A.any_all_pairs = 0;
    A.any_adapt = 0;
    A.nbr_ok = 1;
    for (int k = 0; k < n; ++k) {
        if (table[k].skip) A.any_skip = 1; else A.any_all_pairs = 1;
        if (table[k].kappa > 0.0) A.any_adapt = 1;
        const double dt = std::max(table[k].dt, table[k].dt_max);
        for (int a = 0; a < 3; ++a)
            if (table[k].n[a] > 1 && !(dt <= 0.98 * table[k].dx[a])) A.nbr_ok = 0;
    }
}

int set_small_max(Arena& A, int32_t v)
{
    if (v < 0 || v > 1024) return fail(CUBA_ERR_INVALID, "small_max must lie in [0, 1024]");
    A.small_max = (uint32_t)v;
    return CUBA_OK;
}

// Candidate thresholds of the warp-per-cell path, timed by autotune_arena.
static const int32_t kTuneCandidates[] = {0, 16, 32, 64, 128, 256, 512, 1024};
static const int kTuneCount = (int)(sizeof(kTuneCandidates) / sizeof(kTuneCandidates[0]));

// Time n_steps steps of the arena for every candidate threshold, each from
// the same saved state (positions, momenta, descriptors, counters), then
// restore that state and keep the fastest threshold; with shape_too, then the
// blocks per iteration of the small-cell and the item pair kernel, in that
// order.  The simulations do not advance.  ms (optional) receives the
// timings in candidate order (kTuneCount, then 2 + 3 with shape_too).
static int tune_arena(Arena& A, int n_steps, cudaStream_t st, int32_t* chosen, double* ms, bool shape_too)
{
    if (n_steps < 1) return fail(CUBA_ERR_INVALID, "n_steps must be >= 1");
    if (A.np == 0 || A.nsims == 0) {
        if (chosen) *chosen = (int32_t)A.small_max;
        return CUBA_OK;
    }
    const size_t es = A.precision == CUBA_FP64 ? 8 : 4;
    const size_t col = (size_t)A.np * es;
    void* saved = nullptr;
    int rc = arena_dalloc(A, &saved, 6 * col, "autotune state");
    if (rc) return rc;
    std::vector<SimDesc> table(A.nsims);
    std::vector<unsigned long long> stats((size_t)A.simcap * kStatCount);
    std::vector<uint32_t> cells((size_t)A.ncells + 1);
    CUDA_TRY(cudaDeviceSynchronize(), "sync");
    const int cur0 = A.cur;
    const uint32_t keep = A.small_max;
    for (int c = 0; c < 6; ++c)
        cudaMemcpy((char*)saved + c * col, (char*)A.st[cur0] + (size_t)c * A.pcap * es, col, cudaMemcpyDeviceToDevice);
    cudaMemcpy(table.data(), A.d_sims, table.size() * sizeof(SimDesc), cudaMemcpyDeviceToHost);
    cudaMemcpy(stats.data(), A.stats, stats.size() * 8, cudaMemcpyDeviceToHost);
    cudaMemcpy(cells.data(), A.cell_start, cells.size() * 4, cudaMemcpyDeviceToHost);
    auto restore = [&]() {
        A.cur = cur0;
        for (int c = 0; c < 6; ++c)
            cudaMemcpy((char*)A.st[cur0] + (size_t)c * A.pcap * es, (char*)saved + c * col, col, cudaMemcpyDeviceToDevice);
        cudaMemcpy(A.d_sims, table.data(), table.size() * sizeof(SimDesc), cudaMemcpyHostToDevice);
        cudaMemcpy(A.stats, stats.data(), stats.size() * 8, cudaMemcpyHostToDevice);
        cudaMemcpy(A.cell_start, cells.data(), cells.size() * 4, cudaMemcpyHostToDevice);
        cudaDeviceSynchronize();
    };
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // device time per step of the present shape, from the saved state
    auto time_shape = [&](double* out) -> int {
        restore();
        int r = enqueue_step(A, st);  // warm-up step (also loads the kernels)
        cudaEventRecord(e0, st);
        for (int it = 0; it < n_steps && !r; ++it) r = enqueue_step(A, st);
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        if (!r && e != cudaSuccess) r = cuda_fail(e, "autotune");
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        *out = t / n_steps;
        return r;
    };
    // coordinate 1: small_max
    double best = 1e300;
    int32_t best_v = (int32_t)keep;
    for (int k = 0; k < kTuneCount && !rc; ++k) {
        A.small_max = (uint32_t)kTuneCandidates[k];
        double t = 0.0;
        rc = time_shape(&t);
        if (ms) ms[k] = t;
        if (!rc && t < best) {
            best = t;
            best_v = kTuneCandidates[k];
        }
    }
    A.small_max = rc ? keep : (uint32_t)best_v;
    // coordinates 2 and 3: blocks per iteration of the two pair kernels
    if (shape_too && !rc) {
        const uint32_t small_c[2] = {1u, 2u}, tile_c[3] = {2u, 4u, 8u};
        const uint32_t keep_s = A.small_nb, keep_t = A.tile_nb;
        double bs = 1e300, bt = 1e300;
        uint32_t vs = keep_s, vt = keep_t;
        for (int k = 0; k < 2 && !rc; ++k) {
            A.small_nb = small_c[k];
            double t = 0.0;
            rc = time_shape(&t);
            if (ms) ms[kTuneCount + k] = t;
            if (!rc && t < bs) { bs = t; vs = small_c[k]; }
        }
        A.small_nb = rc ? keep_s : vs;
        for (int k = 0; k < 3 && !rc; ++k) {
            A.tile_nb = tile_c[k];
            double t = 0.0;
            rc = time_shape(&t);
            if (ms) ms[kTuneCount + 2 + k] = t;
            if (!rc && t < bt) { bt = t; vt = tile_c[k]; }
        }
        A.tile_nb = rc ? keep_t : vt;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    restore();
    arena_dfree(A, saved);
    if (chosen) *chosen = (int32_t)A.small_max;
    if (rc) return rc;
    return read_kernel_errors(A);
}

int autotune_arena(Arena& A, int n_steps, cudaStream_t st, int32_t* chosen, double* ms)
{
    return tune_arena(A, n_steps, st, chosen, ms, false);
}

int autotune_shape(Arena& A, int n_steps, cudaStream_t st, cuba_launch_shape* chosen, double* ms)
{
    int32_t sm = 0;
    const int rc = tune_arena(A, n_steps, st, &sm, ms, true);
    if (chosen) get_launch_shape(A, chosen);
    return rc;
}

int set_launch_shape(Arena& A, const cuba_launch_shape* shape)
{
    if (!shape) return fail(CUBA_ERR_INVALID, "shape is NULL");
    if (shape->small_blocks != 1 && shape->small_blocks != 2)
        return fail(CUBA_ERR_INVALID, "small_blocks must be 1 or 2");
    if (shape->tile_blocks != 2 && shape->tile_blocks != 4 && shape->tile_blocks != 8)
        return fail(CUBA_ERR_INVALID, "tile_blocks must be 2, 4 or 8");
    int rc = set_small_max(A, shape->small_max);
    if (rc) return rc;
    A.small_nb = (uint32_t)shape->small_blocks;
    A.tile_nb = (uint32_t)shape->tile_blocks;
    return CUBA_OK;
}

void get_launch_shape(const Arena& A, cuba_launch_shape* shape)
{
    shape->small_max = (int32_t)A.small_max;
    shape->small_blocks = (int32_t)A.small_nb;
    shape->tile_blocks = (int32_t)A.tile_nb;
}

StepGraphs::~StepGraphs()
{
    drop();
    if (capture) cudaStreamDestroy(capture);
}

}  // namespace host
}  // namespace cuba

using namespace cuba::host;

struct cuba_sim {
    cuba_params params;
    SimDesc desc;      // host copy; the step counter lives on the device
    Arena A;
    StepGraphs graphs;
    double* d_obs = nullptr;  // scratch for observables: 2 n_cells doubles + n_cells ints
    double* d_tot = nullptr;  // 4 doubles
};

namespace {

int upload_desc(cuba_sim* s, cudaStream_t st)
{
    CUDA_TRY(cudaMemcpyAsync(s->A.d_sims, &s->desc, sizeof(SimDesc), cudaMemcpyHostToDevice, st), "upload descriptor");
    set_key_param(s->A, &s->desc, 1);
    return CUBA_OK;
}

}  // namespace

extern "C" {

const char* cuba_last_error(void) { return g_last_error.c_str(); }

static int create_sim(const cuba_params* params, int64_t max_particles, const cuba_allocator* mem, cuba_sim** out)
{
    if (!out) return fail(CUBA_ERR_INVALID, "out is NULL");
    *out = nullptr;
    SimDesc S;
    int rc = make_desc(params, &S);
    if (rc) return rc;
    if (max_particles < 0 || max_particles > (int64_t)0x7FFFFFF0) return fail(CUBA_ERR_INVALID, "bad max_particles");
    if (kernels_init()) return fail(CUBA_ERR_CUDA, "kernel attribute setup failed: %s",
                                    cudaGetErrorString(cudaGetLastError()));
    cuba_sim* s = new cuba_sim();
    s->params = *params;
    s->desc = S;
    rc = arena_alloc(s->A, params->precision, (uint32_t)max_particles, S.ncells, 1, mem);
    if (rc) {
        delete s;
        return rc;
    }
    s->A.nsims = 1;
    s->A.ncells = S.ncells;
    s->A.np = 0;
    rc = arena_dalloc(s->A, &s->d_obs, obs_scratch_bytes(S.ncells), "observables");
    if (!rc) rc = arena_dalloc(s->A, &s->d_tot, kTotScratchBytes, "totals");
    if (rc) {
        cuba_destroy(s);
        return rc;
    }
    rc = upload_desc(s, 0);
    if (!rc) {
        cudaError_t e = cudaStreamSynchronize(0);
        if (e != cudaSuccess) rc = cuda_fail(e, "create");
    }
    if (rc) {
        cuba_destroy(s);
        return rc;
    }
    *out = s;
    return CUBA_OK;
}

int cuba_create(const cuba_params* params, int64_t max_particles, cuba_sim** out)
{
    return create_sim(params, max_particles, nullptr, out);
}

int cuba_create_with_allocator(const cuba_params* params, int64_t max_particles, const cuba_allocator* allocator,
                               cuba_sim** out)
{
    if (!allocator || !allocator->alloc || !allocator->free)
        return fail(CUBA_ERR_INVALID, "allocator needs both alloc and free");
    return create_sim(params, max_particles, allocator, out);
}

int64_t cuba_sim_bytes(const cuba_params* params, int64_t max_particles)
{
    SimDesc S;
    if (make_desc(params, &S)) return -1;
    if (max_particles < 0 || max_particles > (int64_t)0x7FFFFFF0) return -1;
    return (int64_t)object_bytes(params->precision, (uint32_t)max_particles, S.ncells, 1);
}

void cuba_destroy(cuba_sim* s)
{
    if (!s) return;
    cudaDeviceSynchronize();
    s->graphs.drop();
    arena_free(s->A);
    delete s;
}

int cuba_init_thermal(cuba_sim* s, int64_t n, const cuba_region* regions, int n_regions, void* stream)
{
    if (!s) return fail(CUBA_ERR_INVALID, "sim is NULL");
    if (n < 0 || n > (int64_t)s->A.pcap)
        return fail(CUBA_ERR_CAPACITY, "n = %lld exceeds max_particles = %u", (long long)n, s->A.pcap);
    cudaStream_t st = (cudaStream_t)stream;
    s->desc.np = (uint32_t)n;
    s->desc.p_off = 0;
    s->desc.cell_off = 0;
    s->desc.step = 0;
    s->A.np = (uint32_t)n;
    int rc = upload_desc(s, st);
    if (!rc) rc = sample_regions(s->A, 0, s->desc, n, regions, n_regions, s->params.L, st);
    if (!rc) rc = settle_arena(s->A, st, nullptr);
    cudaError_t e = cudaStreamSynchronize(st);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "init_thermal");
    return rc;
}

int cuba_init_riemann(cuba_sim* s, int64_t n, double T_left, double T_right, void* stream)
{
    if (!s) return fail(CUBA_ERR_INVALID, "sim is NULL");
    cuba_region R[2];
    const double* L = s->params.L;
    for (int a = 0; a < 3; ++a) {
        R[0].lo[a] = 0.0;
        R[0].hi[a] = L[a];
        R[1].lo[a] = 0.0;
        R[1].hi[a] = L[a];
    }
    R[0].hi[0] = 0.5 * L[0];
    R[1].lo[0] = 0.5 * L[0];
    R[0].T = T_left;
    R[1].T = T_right;
    return cuba_init_thermal(s, n, R, 2, stream);
}

int cuba_init_hotspot(cuba_sim* s, int64_t n, double T0, double dT, double width, void* stream)
{
    if (!s) return fail(CUBA_ERR_INVALID, "sim is NULL");
    if (!(T0 > 0.0) || !(dT >= 0.0) || !(width > 0.0)) return fail(CUBA_ERR_INVALID, "need T0 > 0, dT >= 0, width > 0");
    if (n < 0 || n > (int64_t)s->A.pcap)
        return fail(CUBA_ERR_CAPACITY, "n = %lld exceeds max_particles = %u", (long long)n, s->A.pcap);
    cudaStream_t st = (cudaStream_t)stream;
    s->desc.np = (uint32_t)n;
    s->desc.p_off = 0;
    s->desc.cell_off = 0;
    s->desc.step = 0;
    s->A.np = (uint32_t)n;
    int rc = upload_desc(s, st);
    if (!rc && launch_init_hotspot(s->A, s->desc, T0, dT, width, st))
        rc = fail(CUBA_ERR_CUDA, "hot-spot sampling launch failed");
    if (!rc) rc = settle_arena(s->A, st, nullptr);
    cudaError_t e = cudaStreamSynchronize(st);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "init_hotspot");
    return rc;
}

int cuba_set_state(cuba_sim* s, const void* soa, int64_t n, void* stream)
{
    if (!s || (!soa && n > 0)) return fail(CUBA_ERR_INVALID, "bad arguments");
    if (n < 0 || n > (int64_t)s->A.pcap) return fail(CUBA_ERR_CAPACITY, "n = %lld exceeds max_particles", (long long)n);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = s->A.precision == CUBA_FP64 ? 8 : 4;
    s->A.cur = 0;
    for (int c = 0; c < 6; ++c)
        CUDA_TRY(cudaMemcpyAsync((char*)s->A.st[0] + (size_t)c * s->A.pcap * es, (const char*)soa + (size_t)c * n * es,
                                 (size_t)n * es, cudaMemcpyDefault, st),
                 "copy state in");
    s->desc.np = (uint32_t)n;
    s->desc.p_off = 0;
    s->desc.cell_off = 0;
    // keep the step counter
    uint32_t step = 0;
    CUDA_TRY(cudaMemcpyAsync(&step, &s->A.d_sims[0].step, 4, cudaMemcpyDeviceToHost, st), "read step");
    CUDA_TRY(cudaStreamSynchronize(st), "sync");
    s->desc.step = step;
    s->A.np = (uint32_t)n;
    int rc = upload_desc(s, st);
    if (!rc) rc = settle_arena(s->A, st, nullptr);
    cudaError_t e = cudaStreamSynchronize(st);
    if (!rc && e != cudaSuccess) rc = cuda_fail(e, "set_state");
    return rc;
}

int cuba_get_state(cuba_sim* s, void* out, void* stream)
{
    if (!s || (!out && s->A.np)) return fail(CUBA_ERR_INVALID, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t es = s->A.precision == CUBA_FP64 ? 8 : 4;
    const size_t n = s->A.np;
    for (int c = 0; c < 6; ++c)
        CUDA_TRY(cudaMemcpyAsync((char*)out + (size_t)c * n * es, (const char*)s->A.st[s->A.cur] + (size_t)c * s->A.pcap * es,
                                 n * es, cudaMemcpyDefault, st),
                 "copy state out");
    CUDA_TRY(cudaStreamSynchronize(st), "sync");
    return read_kernel_errors(s->A);
}

int cuba_sizes(const cuba_sim* s, int64_t* np, int64_t* nc)
{
    if (!s) return fail(CUBA_ERR_INVALID, "sim is NULL");
    if (np) *np = s->A.np;
    if (nc) *nc = s->A.ncells;
    return CUBA_OK;
}

int cuba_get_step(const cuba_sim* s, uint32_t* step)
{
    if (!s || !step) return fail(CUBA_ERR_INVALID, "bad arguments");
    CUDA_TRY(cudaMemcpy(step, &s->A.d_sims[0].step, 4, cudaMemcpyDeviceToHost), "read step");
    return CUBA_OK;
}

int cuba_set_step(cuba_sim* s, uint32_t step)
{
    if (!s) return fail(CUBA_ERR_INVALID, "sim is NULL");
    if (step == 0xFFFFFFFFu) return fail(CUBA_ERR_INVALID, "step 0xFFFFFFFF is reserved for sampling");
    CUDA_TRY(cudaDeviceSynchronize(), "sync");
    CUDA_TRY(cudaMemcpy(&s->A.d_sims[0].step, &step, 4, cudaMemcpyHostToDevice), "write step");
    s->desc.step = step;
    return CUBA_OK;
}

int cuba_get_time(const cuba_sim* s, double* time, double* last_dt)
{
    if (!s) return fail(CUBA_ERR_INVALID, "sim is NULL");
    double v[2];
    CUDA_TRY(cudaMemcpy(&v[0], &s->A.d_sims[0].time, sizeof(double), cudaMemcpyDeviceToHost), "read time");
    CUDA_TRY(cudaMemcpy(&v[1], &s->A.d_sims[0].dt, sizeof(double), cudaMemcpyDeviceToHost), "read dt");
    if (time) *time = v[0];
    if (last_dt) *last_dt = v[1];
    return CUBA_OK;
}

int cuba_step(cuba_sim* s, int n_steps, void* stream)
{
    if (!s || n_steps < 0) return fail(CUBA_ERR_INVALID, "bad arguments");
    return s->graphs.run(s->A, n_steps, (cudaStream_t)stream);
}

int cuba_step_profiled(cuba_sim* s, int n_steps, double* phase_ms, void* stream)
{
    if (!s || n_steps < 0 || !phase_ms) return fail(CUBA_ERR_INVALID, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t ev[7];
    for (int k = 0; k < 7; ++k) CUDA_TRY(cudaEventCreate(&ev[k]), "event");
    for (int k = 0; k < 6; ++k) phase_ms[k] = 0.0;
    Arena& A = s->A;
    int rc = CUBA_OK;
    for (int it = 0; it < n_steps && !rc; ++it) {
        cudaEventRecord(ev[0], st);
        if (A.any_adapt && launch_adapt_dt(A, st)) rc = fail(CUBA_ERR_CUDA, "adaptive dt launch failed");
        if (!rc && (nbr_path(A) ? launch_step_nbr(A, st, ev[1]) : launch_step_bin(A, st, ev[1])))
            rc = fail(CUBA_ERR_CUDA, "stream/sort launch failed");
        cudaEventRecord(ev[2], st);
        if (!rc && launch_cell_prep(A, st)) rc = fail(CUBA_ERR_CUDA, "cell preparation launch failed");
        cudaEventRecord(ev[3], st);
        if (!rc && launch_pair_tile(A, st)) rc = fail(CUBA_ERR_CUDA, "pair tile launch failed");
        cudaEventRecord(ev[4], st);
        if (!rc && launch_resolve(A, st)) rc = fail(CUBA_ERR_CUDA, "resolve launch failed");
        cudaEventRecord(ev[5], st);
        if (!rc && launch_advance(A, st)) rc = fail(CUBA_ERR_CUDA, "advance launch failed");
        cudaEventRecord(ev[6], st);
        cudaError_t e = cudaEventSynchronize(ev[6]);
        if (!rc && e != cudaSuccess) rc = cuda_fail(e, "profiled step");
        for (int k = 0; k < 6 && !rc; ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            phase_ms[k] += ms;
        }
    }
    for (int k = 0; k < 7; ++k) cudaEventDestroy(ev[k]);
    if (rc) return rc;
    return read_kernel_errors(s->A);
}

int cuba_set_small_max(cuba_sim* s, int32_t small_max)
{
    if (!s) return fail(CUBA_ERR_INVALID, "sim is NULL");
    CUDA_TRY(cudaDeviceSynchronize(), "sync");
    return set_small_max(s->A, small_max);
}

int cuba_get_small_max(const cuba_sim* s, int32_t* small_max)
{
    if (!s || !small_max) return fail(CUBA_ERR_INVALID, "bad arguments");
    *small_max = (int32_t)s->A.small_max;
    return CUBA_OK;
}

int cuba_set_launch_shape(cuba_sim* s, const cuba_launch_shape* shape)
{
    if (!s) return fail(CUBA_ERR_INVALID, "sim is NULL");
    CUDA_TRY(cudaDeviceSynchronize(), "sync");
    return set_launch_shape(s->A, shape);
}

int cuba_get_launch_shape(const cuba_sim* s, cuba_launch_shape* shape)
{
    if (!s || !shape) return fail(CUBA_ERR_INVALID, "bad arguments");
    get_launch_shape(s->A, shape);
    return CUBA_OK;
}

int cuba_autotune_shape(cuba_sim* s, int n_steps, cuba_launch_shape* chosen, double* ms_per_candidate, void* stream)
{
    if (!s) return fail(CUBA_ERR_INVALID, "sim is NULL");
    return autotune_shape(s->A, n_steps, (cudaStream_t)stream, chosen, ms_per_candidate);
}

int cuba_autotune(cuba_sim* s, int n_steps, int32_t* chosen, double* ms_per_candidate, void* stream)
{
    if (!s) return fail(CUBA_ERR_INVALID, "sim is NULL");
    return autotune_arena(s->A, n_steps, (cudaStream_t)stream, chosen, ms_per_candidate);
}

int cuba_observables(cuba_sim* s, double* T00, double* T0x, int32_t* counts, void* stream)
{
    if (!s) return fail(CUBA_ERR_INVALID, "sim is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t nc = s->A.ncells;
    double* dT00 = s->d_obs;
    double* dT0x = s->d_obs + nc;
    int32_t* dcnt = reinterpret_cast<int32_t*>(s->d_obs + 2 * nc);
    if (launch_observables(s->A, 0, dT00, dT0x, dcnt, st)) return fail(CUBA_ERR_CUDA, "observables launch failed");
    if (T00) CUDA_TRY(cudaMemcpyAsync(T00, dT00, nc * 8, cudaMemcpyDefault, st), "copy T00");
    if (T0x) CUDA_TRY(cudaMemcpyAsync(T0x, dT0x, nc * 8, cudaMemcpyDefault, st), "copy T0x");
    if (counts) CUDA_TRY(cudaMemcpyAsync(counts, dcnt, nc * 4, cudaMemcpyDefault, st), "copy counts");
    CUDA_TRY(cudaStreamSynchronize(st), "sync");
    return read_kernel_errors(s->A);
}

int cuba_totals(cuba_sim* s, double out[4], int64_t* n, void* stream)
{
    if (!s || !out) return fail(CUBA_ERR_INVALID, "bad arguments");
    cudaStream_t st = (cudaStream_t)stream;
    if (launch_totals(s->A, 0, s->d_tot, st)) return fail(CUBA_ERR_CUDA, "totals launch failed");
    CUDA_TRY(cudaMemcpyAsync(out, s->d_tot, 4 * sizeof(double), cudaMemcpyDefault, st), "copy totals");
    CUDA_TRY(cudaStreamSynchronize(st), "sync");
    if (n) *n = s->A.np;
    return read_kernel_errors(s->A);
}

int cuba_stats(cuba_sim* s, cuba_counters* out)
{
    if (!s || !out) return fail(CUBA_ERR_INVALID, "bad arguments");
    unsigned long long h[kStatCount];
    CUDA_TRY(cudaDeviceSynchronize(), "sync");
    CUDA_TRY(cudaMemcpy(h, s->A.stats, sizeof(h), cudaMemcpyDeviceToHost), "read stats");
    out->steps = (int64_t)h[kStatSteps];
    out->pair_tests = (int64_t)h[kStatPairTests];
    out->accepted = (int64_t)h[kStatAccepted];
    out->executed = (int64_t)h[kStatExecuted];
    out->reflections = (int64_t)h[kStatReflections];
    out->fp64_boosts = (int64_t)h[kStatFp64Boosts];
    out->overflow = (int64_t)h[kStatOverflow];
    out->candidates = (int64_t)h[kStatCandidates];
    return read_kernel_errors(s->A);
}

int cuba_trace_enable(cuba_sim* s, int on)
{
    if (!s) return fail(CUBA_ERR_INVALID, "sim is NULL");
    CUDA_TRY(cudaDeviceSynchronize(), "sync");
    if (on && !s->A.trace_keys) {
        int rc = arena_dalloc(s->A, &s->A.trace_keys, (size_t)std::max<uint32_t>(s->A.pcap, 1) * 4, "trace");
        if (rc) return rc;
    }
    s->A.trace = on ? 1 : 0;
    s->graphs.drop();
    return CUBA_OK;
}

int cuba_trace_get(cuba_sim* s, uint32_t* keys, uint32_t* perm, uint32_t* cell_start, uint32_t* pairs,
                   uint8_t* executed, int64_t cap, int64_t* n_pairs)
{
    if (!s) return fail(CUBA_ERR_INVALID, "sim is NULL");
    if (!s->A.trace) return fail(CUBA_ERR_INVALID, "tracing is off");
    CUDA_TRY(cudaDeviceSynchronize(), "sync");
    const Arena& A = s->A;
    const size_t n = A.np, nc = A.ncells;
    if (keys) CUDA_TRY(cudaMemcpy(keys, A.trace_keys, n * 4, cudaMemcpyDeviceToHost), "copy keys");
    if (perm) CUDA_TRY(cudaMemcpy(perm, A.idx[A.sorted_buf], n * 4, cudaMemcpyDeviceToHost), "copy perm");
    if (cell_start) CUDA_TRY(cudaMemcpy(cell_start, A.cell_start, (nc + 1) * 4, cudaMemcpyDeviceToHost), "copy cells");
    std::vector<uint2> work(nc + 1);
    std::vector<uint32_t> cnt(nc);
    CUDA_TRY(cudaMemcpy(work.data(), A.cell_work, (nc + 1) * sizeof(uint2), cudaMemcpyDeviceToHost), "copy work");
    CUDA_TRY(cudaMemcpy(cnt.data(), A.acc_count, nc * 4, cudaMemcpyDeviceToHost), "copy counts");
    int64_t total = 0;
    std::vector<unsigned long long> seg;
    for (size_t c = 0; c < nc; ++c) {
        uint32_t m = std::min(cnt[c], work[c + 1].y - work[c].y);
        if (!m) continue;
        seg.resize(m);
        CUDA_TRY(cudaMemcpy(seg.data(), A.acc + work[c].y, m * 8, cudaMemcpyDeviceToHost), "copy pairs");
        for (uint32_t k = 0; k < m; ++k) {
            if (total < cap) {
                if (pairs) {
                    pairs[3 * total] = (uint32_t)c;
                    pairs[3 * total + 1] = (uint32_t)(seg[k] >> 32) & 0x7FFFFFFFu;
                    pairs[3 * total + 2] = (uint32_t)seg[k];
                }
                if (executed) executed[total] = (seg[k] >> 63) ? 1 : 0;
            }
            ++total;
        }
    }
    if (n_pairs) *n_pairs = total;
    return read_kernel_errors(s->A);
}

int cuba_kinematics_fp32(const float* pin, int64_t npairs, uint64_t key, uint32_t step, double gamma_fp64, float* pout,
                         int32_t* used_fp64, void* stream)
{
    if (npairs < 0 || (npairs > 0 && (!pin || !pout || !used_fp64))) return fail(CUBA_ERR_INVALID, "bad arguments");
    if (npairs > (int64_t)1 << 30) return fail(CUBA_ERR_INVALID, "too many pairs");
    SimDesc S;
    std::memset(&S, 0, sizeof(S));
    S.key0 = (uint32_t)key;
    S.key1 = (uint32_t)(key >> 32);
    S.step = step;
    S.gamma_fp64 = (float)gamma_fp64;
    if (launch_kinematics_check(S, pin, npairs, pout, used_fp64, (cudaStream_t)stream))
        return fail(CUBA_ERR_CUDA, "kinematics launch failed");
    return CUBA_OK;
}

int cuba_philox(const uint32_t* ctr, int64_t n, uint64_t key, uint32_t* out, void* stream)
{
    if (n < 0 || (n > 0 && (!ctr || !out))) return fail(CUBA_ERR_INVALID, "bad arguments");
    if (launch_philox(ctr, n, key, out, (cudaStream_t)stream)) return fail(CUBA_ERR_CUDA, "philox launch failed");
    return CUBA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Binning without allocation
// ---------------------------------------------------------------------------
// Scratch of cuba_bin_noalloc: a file-scope device array of fixed size that
// every GPU loading the library holds until exit.  Layout in 32-bit words:
// keys (2 x max), permutation ping-pong (2 x max), radix histogram
// (256 x tiles), scan partial sums.
namespace {
constexpr uint32_t kNoallocMax = CUBA_NOALLOC_MAX_PARTICLES;
constexpr uint32_t kNoallocTiles = (kNoallocMax + kSortTile - 1) / kSortTile;
constexpr size_t kNoallocPartialWords = 1024;
constexpr size_t kNoallocWords = 4ull * kNoallocMax + (size_t)kRadixBins * kNoallocTiles + kNoallocPartialWords;
}  // namespace

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoallocWords];

namespace {
constexpr int kNoallocMaxDevices = 64;
std::mutex g_noalloc_mutex;
uint32_t* g_noalloc_ptr[kNoallocMaxDevices] = {};

// Device address of the scratch array on the current device; looked up once
// per device (the host-side name of the array is not a device address).
int noalloc_scratch(uint32_t** out)
{
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(CUBA_ERR_INVALID, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress(noalloc scratch)");
        g_noalloc_ptr[dev] = static_cast<uint32_t*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return CUBA_OK;
}
}  // namespace

extern "C" int cuba_bin_noalloc(const cuba_params* params, const void* xyz, int64_t n, uint32_t* perm,
                                uint32_t* cell_start, void* stream)
{
    SimDesc S;
    int rc = make_desc(params, &S);
    if (rc) return rc;
    if (n < 0) return fail(CUBA_ERR_INVALID, "n must be >= 0");
    if (n > (int64_t)kNoallocMax)
        return fail(CUBA_ERR_CAPACITY, "cuba_bin_noalloc handles at most %u particles (got %lld)", kNoallocMax,
                    (long long)n);
    if (!cell_start || (n > 0 && (!xyz || !perm))) return fail(CUBA_ERR_INVALID, "NULL buffer");
    uint32_t* scratch = nullptr;
    rc = noalloc_scratch(&scratch);
    if (rc) return rc;
    const uint32_t m = kNoallocMax;
    uint32_t* key_a = scratch;
    uint32_t* key_b = scratch + m;
    uint32_t* idx_a = scratch + 2ull * m;
    uint32_t* idx_b = scratch + 3ull * m;
    uint32_t* hist = scratch + 4ull * m;
    void* partials = scratch + 4ull * m + (size_t)kRadixBins * kNoallocTiles;
    S.np = (uint32_t)n;
    if (launch_bin_raw(S, params->precision, xyz, (uint32_t)n, key_a, key_b, idx_a, idx_b, hist, partials,
                       kNoallocPartialWords * sizeof(uint32_t), perm, cell_start, (cudaStream_t)stream))
        return fail(CUBA_ERR_CUDA, "binning launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return CUBA_OK;
}
