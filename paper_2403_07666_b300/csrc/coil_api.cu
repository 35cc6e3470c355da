// C ABI of the coil stepper: handle life cycle, validation, host-side
// geometry tables, operator assembly and the per-step launch sequence.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <algorithm>
#include <atomic>
#include <vector>

#include "../../include/coil.h"
#include "common.cuh"
#include "toeplitz_tc.h"

namespace cq {
cudaError_t upload_gl_rule(const double* x, const double* w);
cudaError_t launch_table(const double* rc, const double* zc, const double* hc, int C, int NT,
                         double pitch_t, double* tab, cudaStream_t s);
cudaError_t launch_expand(const double* tab, int C, int NT, int wire_div, long long N, long long ld,
                          int prec, void* M, cudaStream_t s);
cudaError_t launch_near_blocks(const double* tab, int C, int NT, int B, int n_types, double* near,
                               float* nearf, cudaStream_t s);
cudaError_t launch_gemv(const CoilDev* cds, int n_coils, int prec, long long max_rows, int which,
                        int n_sm, cudaStream_t s);
size_t toeplitz_part_floats(int C, int NT);
cudaError_t launch_toeplitz_table(const double* tab, int C, int NT, int wire_div, float* out, cudaStream_t s);
cudaError_t launch_toeplitz(const CoilDev* cds, int n_coils, int max_C, int max_NT, long long max_N, int n_sm,
                            cudaStream_t s);

__global__ void k_pointwise(const CoilDev* __restrict__ cds);
__global__ void k_factor(const CoilDev* __restrict__ cds);
__global__ void k_factor_med(const CoilDev* __restrict__ cds, int fuse_scale);
__global__ void k_init_med(const CoilDev* __restrict__ cds, int fuse_init);
__global__ void k_update_med(const CoilDev* __restrict__ cds, int fuse_beta, cudaGraphConditionalHandle cond,
                             int use_cond);
__global__ void k_near_med(const CoilDev* __restrict__ cds, int which, int far_tiles, int fuse_alpha);
__global__ void k_near(const CoilDev* __restrict__ cds, int which);
__global__ void k_init(const CoilDev* __restrict__ cds);
__global__ void k_update(const CoilDev* __restrict__ cds);
__global__ void k_near_seg(const CoilDev* __restrict__ cds, int which, int far_tiles, int fuse_alpha,
                           int near_pre);
__global__ void k_init_seg(const CoilDev* __restrict__ cds, int fuse_init, int fuse_near, int far_tiles, int near_pre);
__global__ void k_update_seg(const CoilDev* __restrict__ cds, int fuse_beta, cudaGraphConditionalHandle cond,
                             int use_cond);
__global__ void k_pointwise_seg(const CoilDev* __restrict__ cds);
__global__ void k_factor_seg(const CoilDev* __restrict__ cds, int fuse_scale);
__global__ void k_factor_seg_groups(const CoilDev* __restrict__ cds);
__global__ void k_direction(const CoilDev* __restrict__ cds);
__global__ void k_reduce(const CoilDev* __restrict__ cds, int mode, int skip_seg);
__global__ void k_finalize(const CoilDev* __restrict__ cds);
__global__ void k_replay_restore(const CoilDev* __restrict__ cds);
__global__ void k_finalize_seg(const CoilDev* __restrict__ cds);
__global__ void k_adi_r(const CoilDev* __restrict__ cds);
cudaError_t adi_allow_smem(size_t bytes);
cudaError_t adj_adi_allow_smem(size_t bytes);
__global__ void k_adi_z(const CoilDev* __restrict__ cds);
__global__ void k_step_end(const CoilDev* __restrict__ cds);
__global__ void k_read(const CoilDev* __restrict__ cds, double Ba, double* J, double* Br, double* Bz,
                       double* T);
__global__ void k_moment(const CoilDev* __restrict__ cds, double* part);
__global__ void k_moment_sum(const double* part, int n, double* out);
__global__ void k_to_float(const double* x, float* f, int n);
__global__ void k_gather_status(const CoilDev* __restrict__ cds, int n, int* out);
__global__ void k_loop_cond(const CoilDev* __restrict__ cds, cudaGraphConditionalHandle h);
__global__ void k_batch_cond(const CoilDev* __restrict__ cds, int n, int* passes, int maxit,
                             cudaGraphConditionalHandle h);
}  // namespace cq

// A batched step captured as one graph, kept by the batch's first coil for the
// next call with the same coils (matched by their creation ids).
struct BatchGraph {
    std::vector<long long> ids;
    cq::CoilDev* dd = nullptr;    // n descriptors, then 3 n + 1 ints: done, status, iter per coil; passes
    int* hstat = nullptr;         // pinned copy of the 3 n + 1 ints
    cudaGraphExec_t exec = nullptr;
    int fixed = 0, per_pass = 0;
};

using namespace cq;

struct coil {
    int device = 0;
    int n_sm = 148;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    CoilDev h{};                 // host copy of the descriptor
    CoilDev* d = nullptr;        // device copy
    Scalars* pinned = nullptr;   // host-pinned mirror of the device scalars
    std::vector<void*> allocs;
    size_t bytes = 0;
    size_t op_bytes = 0;
    std::string err;
    // host copies needed later
    std::vector<double> r_host, area_host, Kr_host, Kz_host;
    int n_sub = 0, gap_kind = 0;
    double thomas_dt = -1.0;
    long long steps = 0;
    double t = 0.0;
    int last_iters = 8;
    double setup_ms = 0.0;
    coil_drive drive{};
    bool has_drive = false;
    double* readbuf = nullptr;   // 5 N doubles for coil_read + moment partials
    // counters and optional operator timing
    int profile = 0;
    long long launches = 0, op_launches = 0, pcg_iters = 0;
    double op_ms = 0.0;
    std::vector<cudaEvent_t> ev_pool;
    // side streams and their events for the batched tensor-core applies
    std::vector<cudaStream_t> aux;
    std::vector<cudaEvent_t> aux_ev;
    // the step as one graph (prologue, PCG while loop, epilogue, scalars read
    // back), when operator applies are not being timed one by one
    cudaGraphExec_t step_exec = nullptr;
    cudaStream_t body_stream = nullptr;
    bool graph_failed = false;
    int graph_fixed = 0, graph_per_pass = 0;   // kernels outside and inside the loop
    // the adjoint's transposed solve as one graph (its prologue and PCG loop)
    cudaGraphExec_t adj_exec = nullptr;
    int adj_fixed = 0, adj_per_pass = 0;
    // the adjoint's replayed forward step as one graph (no solve)
    cudaGraphExec_t replay_exec = nullptr;
    int replay_fixed = 0;
    long long uid = 0;           // creation id (batched-step graphs match coils by it)
    BatchGraph* batch = nullptr;
    size_t ev_used = 0;          // event pairs recorded since the last harvest
    cq::TcPlan* tc = nullptr;    // tensor-core Toeplitz apply (format 2)
    // the first coil of a batch keeps the batch's one-launch tensor-core
    // applies (the coils' arguments) for that set of coils
    cq::TcBatch* tcb = nullptr;
    std::vector<long long> tcb_ids;
};

namespace {

const char* kNoHandle = "null coil handle";
constexpr int kAuxStreams = 16;         // side streams of a batch's tensor-core applies
constexpr int kRedThreads = 1024;       // threads of the one-CTA-per-coil reductions (k_reduce, k_step_end)
constexpr size_t kMomentBlocks = 148;   // partial sums of the moment in coil_read

std::string tc_timeout_text(const coil_t* c);

coil_status fail(coil_t* c, coil_status st, const std::string& msg) {
    if (c) c->err = msg;
    return st;
}

coil_status reset_wire_stats(coil_t* c, bool onsets);
coil_status read_scalars(coil_t* c);

// "tensor-core apply timed out", with the first wait that ran out when the
// apply recorded one (site, CTA, stage, index, parity, thread)
std::string tc_timeout_text(const coil_t* c) {
    std::string s = "tensor-core apply timed out";
    const int* w = c->pinned ? c->pinned->tc_where : nullptr;
    if (w && w[0] != 0) {
        s += " (wait site " + std::to_string(w[0]) + ", CTA " + std::to_string(w[1]) + ", stage " +
             std::to_string(w[2]) + ", index " + std::to_string(w[3]) + ", parity " + std::to_string(w[4]) +
             ", thread " + std::to_string(w[5]) + ")";
        if (c->tc && c->tc->prog && w[1] >= 0 && w[1] < c->tc->sh.n_cta) {
            int pr[32];
            if (cudaMemcpy(pr, c->tc->prog + 32 * w[1], sizeof(pr), cudaMemcpyDeviceToHost) == cudaSuccess) {
                s += " progress:";
                for (int k = 0; k < 24; ++k) s += " " + std::to_string(pr[k]);
            }
        }
    }
    return s;
}
coil_status sync_descriptor(coil_t* c);

coil_status cuda_fail(coil_t* c, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(c, COIL_ERR_OOM, m);
    return fail(c, COIL_ERR_CUDA, m);
}

#define CK(call, where)                                   \
    do {                                                  \
        cudaError_t e__ = (call);                         \
        if (e__ != cudaSuccess) return cuda_fail(c, e__, where); \
    } while (0)

template <typename T>
coil_status dalloc(coil_t* c, T** p, size_t count, const char* what) {
    size_t nb = count * sizeof(T);
    if (nb == 0) nb = 16;
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, nb);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, COIL_ERR_OOM, std::string("device allocation of ") + what + " failed (" +
                                         std::to_string(nb) + " bytes)");
    }
    c->allocs.push_back(v);
    c->bytes += nb;
    *p = static_cast<T*>(v);
    CK(cudaMemsetAsync(v, 0, nb, c->stream), "memset");
    return COIL_OK;
}

template <typename T>
coil_status upload(coil_t* c, T** p, const std::vector<T>& host, const char* what) {
    coil_status st = dalloc(c, p, host.size(), what);
    if (st != COIL_OK) return st;
    if (!host.empty())
        CK(cudaMemcpyAsync(*p, host.data(), host.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream),
           what);
    return COIL_OK;
}

#define TRY(x)                               \
    do {                                     \
        coil_status s__ = (x);               \
        if (s__ != COIL_OK) return s__;      \
    } while (0)

bool is_fin(double v) { return isfinite(v) != 0; }

// FP32 copies of the material constants (round to nearest, as a device
// conversion would give).
void round_constants(CoilDev& h) {
    h.f_E0 = (float)h.E0; h.f_nexp = (float)h.nexp; h.f_Jc0 = (float)h.Jc0; h.f_Tc = (float)h.Tc;
    h.f_Bc2_0 = (float)h.Bc2_0; h.f_B_reg = (float)h.B_reg; h.f_C_eps = (float)h.C_eps;
    h.f_p_eps = (float)h.p_eps; h.f_rho_n = (float)h.rho_n; h.f_T_bath = (float)h.T_bath;
}

// 3-point Lagrange derivative weights at x for nodes x0 < x1 < x2.
void lagrange_weights(double x0, double x1, double x2, double x, double* w) {
    w[0] = ((x - x1) + (x - x2)) / ((x0 - x1) * (x0 - x2));
    w[1] = ((x - x0) + (x - x2)) / ((x1 - x0) * (x1 - x2));
    w[2] = ((x - x0) + (x - x1)) / ((x2 - x0) * (x2 - x1));
}

void stencil_axis(const std::vector<double>& ax, std::vector<int>& j0, std::vector<double>& w) {
    int G = (int)ax.size();
    j0.assign(G, 0);
    w.assign(3 * (size_t)G, 0.0);
    for (int k = 0; k < G; ++k) {
        if (G >= 3) {
            int j = k - 1;
            if (j < 0) j = 0;
            if (j > G - 3) j = G - 3;
            j0[k] = j;
            lagrange_weights(ax[j], ax[j + 1], ax[j + 2], ax[k], &w[3 * (size_t)k]);
        } else if (G == 2) {
            double s = 1.0 / (ax[1] - ax[0]);
            w[3 * (size_t)k] = -s;
            w[3 * (size_t)k + 1] = s;
        }
    }
}

// Thomas factors of (I - hd/C A) for face conductances K (G - 1 faces).
// Thomas factors of (I - hd/C A) on one grid line (A the conductance
// Laplacian with link conductances K), in the recurrence form of the line
// solve: forward y_i = lo_i y_{i-1} + inv_i v_i, backward x_i = cp_i x_{i+1} +
// y_i (on return lo holds the forward coefficients -l_i / d_i and cp the
// backward ones -u_i / d_i; lo_0 = cp_{G-1} = 0).
void thomas_factors(const std::vector<double>& K, double hd, double C, std::vector<double>& lo,
                    std::vector<double>& inv, std::vector<double>& cp) {
    int G = (int)K.size() + 1;
    std::vector<double> diag(G, 1.0), up(G, 0.0);
    lo.assign(G, 0.0);
    double cf = hd / C;
    for (int i = 0; i + 1 < G; ++i) {
        lo[i + 1] = -cf * K[i];
        up[i] = -cf * K[i];
        diag[i] += cf * K[i];
        diag[i + 1] += cf * K[i];
    }
    inv.assign(G, 0.0);
    cp.assign(G, 0.0);
    double den = diag[0];
    inv[0] = 1.0 / den;
    cp[0] = G > 1 ? up[0] / den : 0.0;
    for (int i = 1; i < G; ++i) {
        den = diag[i] - lo[i] * cp[i - 1];
        inv[i] = 1.0 / den;
        cp[i] = (i < G - 1) ? up[i] / den : 0.0;
    }
    for (int i = 0; i < G; ++i) {
        lo[i] = i > 0 ? -lo[i] * inv[i] : 0.0;
        cp[i] = i < G - 1 ? -cp[i] : 0.0;
    }
}

double host_drive_field(const coil_drive* d, double t) {
    if (!d || d->Ba_waveform == 0 || d->Ba_rate == 0.0) return 0.0;
    if (d->Ba_waveform == 1) return fmin(d->Ba_rate * t, d->Ba_max);
    double period = 4.0 * d->Ba_max / d->Ba_rate;
    double tau = t - period * floor(t / period);
    if (tau < 0.25 * period) return d->Ba_rate * tau;
    if (tau < 0.75 * period) return d->Ba_max - d->Ba_rate * (tau - 0.25 * period);
    return -d->Ba_max + d->Ba_rate * (tau - 0.75 * period);
}

coil_status validate(const coil_geometry* g, const coil_material* m, const coil_options* o, coil_t* c) {
    if (!g || !m || !o) return fail(c, COIL_ERR_INVALID, "null geometry, material or options");
    if (o->precision < 0 || o->precision > 2) return fail(c, COIL_ERR_INVALID, "unknown precision");
    if (!(o->rtol > 0.0 && o->rtol < 1.0)) return fail(c, COIL_ERR_INVALID, "rtol must be in (0, 1)");
    if (o->maxit < 1) return fail(c, COIL_ERR_INVALID, "maxit must be >= 1");
    if (o->format != COIL_FORMAT_DENSE && o->format != COIL_FORMAT_TOEPLITZ && o->format != COIL_FORMAT_TOEPLITZ_TC)
        return fail(c, COIL_ERR_INVALID, "unknown operator format");
    if (o->format != COIL_FORMAT_DENSE && (g->kind != COIL_GEOM_SOLENOID || o->precision != PREC_FP32))
        return fail(c, COIL_ERR_INVALID, "the Toeplitz formats need a solenoid and FP32 precision");
    if (o->format == COIL_FORMAT_TOEPLITZ_TC && g->n_turns > kTcMaxTurns)
        return fail(c, COIL_ERR_INVALID, "the tensor-core Toeplitz format takes at most 112 turns");
    if (g->kind == COIL_GEOM_SOLENOID) {
        if (g->n_layers < 1 || g->n_turns < 1 || g->n_sub < 1)
            return fail(c, COIL_ERR_INVALID, "solenoid needs n_layers, n_turns, n_sub >= 1");
        if (g->n_sub * g->n_sub > kMaxBlock)
            return fail(c, COIL_ERR_INVALID, "n_sub^2 must not exceed 64 elements per wire");
        if (!(g->wire_d > 0.0) || !(g->pitch >= g->wire_d) || !(g->r_in >= 0.0) || !is_fin(g->pitch) ||
            !is_fin(g->r_in))
            return fail(c, COIL_ERR_INVALID, "solenoid needs wire_d > 0, pitch >= wire_d, r_in >= 0");
        double n_elem = (double)g->n_layers * g->n_turns * g->n_sub * g->n_sub;
        if (n_elem > 2.0e8) return fail(c, COIL_ERR_INVALID, "too many elements");
    } else if (g->kind == COIL_GEOM_LIST) {
        if (g->n_elem < 1 || g->block < 1 || g->block > kMaxBlock || g->n_elem % g->block)
            return fail(c, COIL_ERR_INVALID, "list needs n_elem a multiple of block, 1 <= block <= 64");
        if (!g->r || !g->z || !g->h || !g->block_transport)
            return fail(c, COIL_ERR_INVALID, "list needs r, z, h and block_transport");
        for (int i = 0; i < g->n_elem; ++i) {
            if (!(g->r[i] > 0.0) || !is_fin(g->r[i]) || !is_fin(g->z[i]) || !(g->h[i] > 0.0) ||
                !is_fin(g->h[i]))
                return fail(c, COIL_ERR_NONFINITE, "list element with non-finite or non-positive r/h");
            if (!(g->h[i] < 2.0 * g->r[i])) return fail(c, COIL_ERR_INVALID, "element crosses the axis");
        }
        if (m->thermal || m->jc_model != 1)
            return fail(c, COIL_ERR_INVALID, "list geometry has no grid: needs thermal = 0, jc_model = 1");
    } else {
        return fail(c, COIL_ERR_INVALID, "unknown geometry kind");
    }
    if (g->n_groups > 1) {
        static_assert(COIL_MAX_GROUPS == kGroupMax, "subelement limit of the ABI and the kernels");
        const int B = g->kind == COIL_GEOM_SOLENOID ? g->n_sub * g->n_sub : g->block;
        if (!g->group || g->n_groups > (B <= kSegMax ? kGroupMaxSeg : COIL_MAX_GROUPS))
            return fail(c, COIL_ERR_INVALID,
                        "subelements need a group array and at most 6 groups (blocks of up to 16 elements) or 16");
        std::vector<int> cnt(g->n_groups, 0);
        for (int k = 0; k < B; ++k) {
            if (g->group[k] < 0 || g->group[k] >= g->n_groups)
                return fail(c, COIL_ERR_INVALID, "subelement group id outside [0, n_groups)");
            ++cnt[g->group[k]];
        }
        for (int v : cnt)
            if (!v) return fail(c, COIL_ERR_INVALID, "empty subelement group");
    }
    const double vals[] = {m->E0, m->n, m->Jc0, m->Tc, m->Bc2_0, m->B_reg, m->C_eps, m->p_eps,
                           m->rho_n, m->rho_m, m->c0, m->kappa_cu, m->kappa_ep, m->h0, m->T_ref, m->T_bath};
    for (double v : vals)
        if (!is_fin(v)) return fail(c, COIL_ERR_NONFINITE, "non-finite material constant");
    if (!(m->rho_n > 0.0) || !(m->E0 > 0.0) || !(m->n >= 1.0) || !(m->T_bath > 0.0) || !(m->T_ref > 0.0) ||
        !(m->rho_m > 0.0) || !(m->c0 > 0.0) || !(m->kappa_cu > 0.0) || !(m->kappa_ep > 0.0) ||
        !(m->Tc > 0.0) || !(m->Bc2_0 > 0.0) || !(m->B_reg > 0.0) || m->h0 < 0.0)
        return fail(c, COIL_ERR_INVALID, "material constant out of range");
    if (!m->jc_factor || !m->strain || !m->mat)
        return fail(c, COIL_ERR_INVALID, "jc_factor, strain and mat arrays are required");
    if (!is_fin(m->Y_eff) || m->Y_eff < 0.0) return fail(c, COIL_ERR_INVALID, "Y_eff must be finite and >= 0");
    return COIL_OK;
}

// ---- schedule of the tensor-core apply and its autotuner

// Device buffers of the current schedule (work list, reduction lists, partial
// tiles), freed when another schedule replaces it.
void tc_free_schedule(coil_t* c) {
    TcPlan& P = *c->tc;
    for (void* p : P.sched_bufs) {
        for (size_t i = 0; i < c->allocs.size(); ++i)
            if (c->allocs[i] == p) { c->allocs.erase(c->allocs.begin() + i); break; }
        cudaFree(p);
    }
    c->bytes -= P.sched_bytes;
    P.sched_bufs.clear();
    P.sched_bytes = 0;
    P.part = P.part2 = nullptr;
    P.work = nullptr;
    P.range = P.l1 = P.l2 = nullptr;
    P.segs1 = P.segs2 = P.prog = nullptr;
}

template <typename T>
coil_status tc_sched_alloc(coil_t* c, T** p, size_t count, const std::vector<T>* host, const char* what) {
    const size_t before = c->allocs.size(), b0 = c->bytes;
    TRY(host ? upload(c, p, *host, what) : dalloc(c, p, count, what));
    if (c->allocs.size() > before) {
        c->tc->sched_bufs.push_back(c->allocs.back());
        c->tc->sched_bytes += c->bytes - b0;
    }
    return COIL_OK;
}

// Make `sh` (mode 0: each table tile loaded by the CTAs of both its products;
// mode 1: one-fill) the coil's schedule: work list, reduction lists, partial
// tiles; the descriptor fields that point at them; graphs captured with the
// previous schedule are dropped.
coil_status tc_plan_schedule(coil_t* c, const TcShape& sh) {
    TcPlan& P = *c->tc;
    CoilDev& h = c->h;
    if (c->stream) CK(cudaStreamSynchronize(c->stream), "schedule");
    tc_free_schedule(c);
    P.sh = sh;
    P.smem = tc_smem_bytes(sh);
    const size_t NT = sh.NT;
    std::vector<int4> work;
    if (sh.mode == 1) {
        std::vector<int2> l1, l2;
        std::vector<int> s1, s2;
        tc2_schedule(&P.sh, &work, &l1, &s1, &l2, &s2);
        TRY(tc_sched_alloc(c, &P.part, (size_t)P.sh.n_seg * NT * 128, (const std::vector<float>*)nullptr,
                           "tensor-core partial tiles"));
        TRY(tc_sched_alloc(c, &P.part2, (size_t)P.sh.n_seg * NT * 64, (const std::vector<float>*)nullptr,
                           "tensor-core partial tiles"));
        TRY(tc_sched_alloc(c, &P.work, 0, &work, "tensor-core schedule"));
        TRY(tc_sched_alloc(c, &P.l1, 0, &l1, "tensor-core schedule"));
        TRY(tc_sched_alloc(c, &P.l2, 0, &l2, "tensor-core schedule"));
        TRY(tc_sched_alloc(c, &P.segs1, 0, &s1, "tensor-core schedule"));
        TRY(tc_sched_alloc(c, &P.segs2, 0, &s2, "tensor-core schedule"));
        TRY(tc_sched_alloc(c, &P.prog, (size_t)P.sh.n_cta * 32, (const std::vector<int>*)nullptr,
                           "tensor-core progress"));
    } else {
        std::vector<int2> range;
        tc_schedule(sh, c->n_sm, &work, &range);
        P.sh.n_cta = (int)work.size();
        TRY(tc_sched_alloc(c, &P.part, (size_t)P.sh.n_cta * NT * 128, (const std::vector<float>*)nullptr,
                           "tensor-core partial tiles"));
        TRY(tc_sched_alloc(c, &P.work, 0, &work, "tensor-core schedule"));
        TRY(tc_sched_alloc(c, &P.range, 0, &range, "tensor-core schedule"));
    }
    h.tc_mode = sh.mode;
    h.tc_part = P.part;
    h.tc_part2 = P.part2;
    h.tc_range = P.range;
    h.tc_l1 = P.l1;
    h.tc_l2 = P.l2;
    h.tc_segs1 = P.segs1;
    h.tc_segs2 = P.segs2;
    if (c->d) TRY(sync_descriptor(c));
    if (c->step_exec) { cudaGraphExecDestroy(c->step_exec); c->step_exec = nullptr; }
    if (c->adj_exec) { cudaGraphExecDestroy(c->adj_exec); c->adj_exec = nullptr; }
    if (c->replay_exec) { cudaGraphExecDestroy(c->replay_exec); c->replay_exec = nullptr; }
    if (c->batch) {
        if (c->batch->exec) cudaGraphExecDestroy(c->batch->exec);
        cudaFree(c->batch->dd);
        cudaFreeHost(c->batch->hstat);
        delete c->batch;
        c->batch = nullptr;
    }
    if (c->stream) CK(cudaStreamSynchronize(c->stream), "schedule");
    return COIL_OK;
}

// Schedules the autotuner has chosen, per (device, C, NT, SM count).
struct TcTuned {
    TcShape sh;
    double us;
};
std::mutex g_tune_mutex;
std::map<std::tuple<int, int, int, int>, TcTuned> g_tuned;

// Mean duration of the apply kernel (split excluded) over a few launches on
// the coil's stream, after one untimed launch.
coil_status tc_time_apply(coil_t* c, double* us) {
    TcPlan& P = *c->tc;
    const int kReps = 4;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "tune");
    CK(cudaEventCreate(&e1), "tune");
    CK(cudaMemsetAsync(&c->h.sc->done, 0, sizeof(int), c->stream), "tune");
    CK(launch_tc_split(P, c->stream, false), "tune");
    CK(launch_tc_apply(P, c->stream, false), "tune");
    CK(cudaEventRecord(e0, c->stream), "tune");
    for (int r = 0; r < kReps; ++r) CK(launch_tc_apply(P, c->stream, false), "tune");
    CK(cudaEventRecord(e1, c->stream), "tune");
    CK(cudaStreamSynchronize(c->stream), "tune");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    read_scalars(c);
    if (c->pinned->status == ST_KERNEL) return fail(c, COIL_ERR_CUDA, tc_timeout_text(c));
    *us = 1e3 * ms / kReps;
    return COIL_OK;
}

// Autotuner of the tensor-core apply: time a small grid of schedules (the
// two-fill apply with 6 to 4 table stages; the one-fill apply with its
// largest stage count and with one fewer, on all SMs and on nine tenths of
// them) on this coil's own table, keep the fastest, and remember it for later
// coils of the same shape.  retune: ignore the remembered choice.
coil_status tc_autotune(coil_t* c, bool retune) {
    const TcShape base = c->tc->sh;
    const auto key = std::make_tuple(c->device, base.C, base.NT, c->n_sm);
    if (!retune) {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) {
            c->tc->tuned_us = it->second.us;
            c->tc->tuned_sh = it->second.sh;
            return tc_plan_schedule(c, it->second.sh);
        }
    }
    std::vector<TcShape> cand;
    TcShape s0;
    if (tc_shape(base.C, base.NT, c->n_sm, &s0)) {
        // the two-fill apply: its largest stage count and one fewer, with the
        // step floor per CTA (small coils on few SMs) and without it
        for (int ms : {0, 1})
            for (int drop = 0; drop < 2; ++drop) {
                TcShape s = s0;
                s.min_steps = ms;
                s.stages = s0.stages - drop;
                if (s.stages < 2 || s.n_acc > s.stages) continue;
                s.n_cta = (int)tc_schedule(s, c->n_sm, nullptr, nullptr);
                if (ms == 1 && s.n_cta == s0.n_cta) continue;        // the floor changed nothing
                cand.push_back(s);
            }
    }
    // the one-fill apply: the default CTA count (a stage floor per CTA) and all
    // SMs, its largest stage count and one fewer
    for (int ctas : {0, c->n_sm}) {
        TcShape s1;
        if (!tc2_shape(base.C, base.NT, c->n_sm, ctas, 0, &s1)) continue;
        if (ctas != 0 && !cand.empty() && cand.back().mode == 1 && cand.back().n_cta == s1.n_cta) continue;
        cand.push_back(s1);
        TcShape s2;
        if (s1.stages > 2 && tc2_shape(base.C, base.NT, c->n_sm, ctas, s1.stages - 1, &s2)) cand.push_back(s2);
    }
    double best = 1e300;
    TcShape best_sh = base;
    c->tc->tuned.clear();
    for (const TcShape& sh : cand) {
        TRY(tc_plan_schedule(c, sh));
        double us = 0.0;
        TRY(tc_time_apply(c, &us));
        c->tc->tuned.push_back({sh.mode, c->tc->sh.n_cta, sh.stages, us});
        if (us < best) { best = us; best_sh = c->tc->sh; }
    }
    TRY(tc_plan_schedule(c, best_sh));
    c->tc->tuned_us = best;
    c->tc->tuned_sh = best_sh;
    c->tc->in_batch = false;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tuned[key] = {best_sh, best};
    return COIL_OK;
}

coil_status setup(coil_t* c, const coil_geometry* g, const coil_material* m, const coil_options* o) {
    CoilDev& h = c->h;
    const bool sol = g->kind == COIL_GEOM_SOLENOID;
    int N, B, W, C, NT, n_types;
    double pitch_t;
    std::vector<double> r, z, hh;
    std::vector<int> constrained, block_type;
    std::vector<int> elem_grid, grid_elem;
    int Gr = 0, Gz = 0, n = 0;
    double gap = 0.0, hel = 0.0;
    std::vector<double> r_axis, z_axis;
    if (sol) {
        n = g->n_sub;
        int NL = g->n_layers;
        NT = g->n_turns;
        B = n * n;
        W = NL * NT;
        N = W * B;
        C = NL * B;
        n_types = NL;
        pitch_t = g->pitch;
        gap = g->pitch - g->wire_d;
        hel = g->wire_d / n;
        Gr = NL * n;
        Gz = NT * n;
        r.resize(N);
        z.resize(N);
        hh.assign(N, hel);
        elem_grid.resize(N);
        grid_elem.resize((size_t)Gr * Gz);
        for (int e = 0; e < N; ++e) {
            int a = e % n, b = (e / n) % n, w = e / B, l = w % NL, t = w / NL;
            r[e] = g->r_in + 0.5 * gap + l * g->pitch + (a + 0.5) * hel;
            z[e] = -0.5 * NT * g->pitch + 0.5 * gap + t * g->pitch + (b + 0.5) * hel;
            int ir = l * n + a, iz = t * n + b;
            elem_grid[e] = iz * Gr + ir;
            grid_elem[(size_t)iz * Gr + ir] = e;
        }
        constrained.assign(W, g->transport ? 1 : 0);
        block_type.resize(W);
        for (int w = 0; w < W; ++w) block_type[w] = w % NL;
        r_axis.resize(Gr);
        z_axis.resize(Gz);
        for (int i = 0; i < Gr; ++i) r_axis[i] = r[grid_elem[i]];
        for (int j = 0; j < Gz; ++j) z_axis[j] = z[grid_elem[(size_t)j * Gr]];
        c->n_sub = n;
    } else {
        N = g->n_elem;
        B = g->block;
        W = N / B;
        C = N;
        NT = 1;
        n_types = W;
        pitch_t = 0.0;
        r.assign(g->r, g->r + N);
        z.assign(g->z, g->z + N);
        hh.assign(g->h, g->h + N);
        constrained.resize(W);
        block_type.resize(W);
        for (int w = 0; w < W; ++w) {
            constrained[w] = g->block_transport[w] ? 1 : 0;
            block_type[w] = w;
        }
    }
    for (int e = 0; e < N; ++e) {
        if (!is_fin(m->jc_factor[e]) || !is_fin(m->strain[e]) || m->jc_factor[e] < 0.0)
            return fail(c, COIL_ERR_NONFINITE, "non-finite or negative jc_factor / strain");
        if (m->mat[e] != 0 && m->mat[e] != 1) return fail(c, COIL_ERR_INVALID, "mat must be 0 or 1");
    }
    h.N = N;
    h.W = W;
    h.B = B;
    h.n_types = n_types;
    h.has_grid = sol ? 1 : 0;
    h.Gr = Gr;
    h.Gz = Gz;
    if (sol) {
        // each ADI line solve holds its line and three factor rows in shared memory
        const size_t line_smem = adi_smem_bytes(std::max(Gr, Gz));
        if (line_smem > (size_t)227 * 1024)
            return fail(c, COIL_ERR_INVALID, "thermal grid line longer than 7,264 cells (layers or turns x n_sub)");
        if (line_smem > (size_t)48 * 1024) {
            CK(adi_allow_smem(line_smem), "ADI shared memory");
            CK(adj_adi_allow_smem(line_smem), "ADI shared memory");
        }
    }
    h.thermal = (sol && m->thermal) ? 1 : 0;
    h.jc_model = m->jc_model;
    h.precision = o->precision;
    h.ld = ((long long)N + 63) / 64 * 64;
    h.E0 = m->E0; h.nexp = m->n; h.Jc0 = m->Jc0; h.Tc = m->Tc; h.Bc2_0 = m->Bc2_0; h.B_reg = m->B_reg;
    h.inv_Y = m->Y_eff > 0.0 ? 1.0 / m->Y_eff : 0.0;
    h.lorentz = h.inv_Y > 0.0 ? 1 : 0;
    h.C_eps = m->C_eps; h.p_eps = m->p_eps; h.rho_n = m->rho_n; h.rho_m = m->rho_m; h.c0 = m->c0;
    h.h0 = m->h0; h.T_ref = m->T_ref; h.T_bath = m->T_bath;
    h.u_bath = h.T_bath * h.T_bath * h.T_bath * h.T_bath;
    round_constants(h);
    h.maxit = o->maxit;
    h.rtol2 = o->rtol * o->rtol;
    h.diag_cap = o->diag_capacity > 0 ? o->diag_capacity : 65536;

    std::vector<double> area(N);
    for (int e = 0; e < N; ++e) area[e] = hh[e] * hh[e];
    c->r_host = r;
    c->area_host = area;
    std::vector<double> jf(m->jc_factor, m->jc_factor + N), st(m->strain, m->strain + N);
    std::vector<int> mt(m->mat, m->mat + N);
    double* dp;
    int* ip;
    TRY(upload(c, &dp, r, "r")); h.r = dp;
    TRY(upload(c, &dp, area, "area")); h.area = dp;
    TRY(upload(c, &dp, jf, "jc_factor")); h.jc_factor = dp;
    TRY(upload(c, &dp, st, "strain")); h.strain = dp;
    std::vector<double> stp(N);
    for (int e = 0; e < N; ++e) stp[e] = pow(fabs(st[e]), m->p_eps);
    TRY(upload(c, &dp, stp, "strain power")); h.strain_pow = dp;
    {
        std::vector<float4> geo(N);
        std::vector<float> spf(N);
        std::vector<double> pr2(N);
        for (int e = 0; e < N; ++e) {
            const float tpr = 2.0f * (float)kPi * (float)r[e];
            const float a = (float)area[e];
            geo[e] = make_float4(tpr, 1.0f / tpr, a, 1.0f / a);
            spf[e] = (float)stp[e];
            pr2[e] = kPi * r[e] * r[e];
        }
        float4* gp;
        float* fp;
        TRY(upload(c, &gp, geo, "geometry (FP32)")); h.geo_f = gp;
        TRY(upload(c, &fp, spf, "strain power (FP32)")); h.strain_pow_f = fp;
        TRY(upload(c, &dp, pr2, "pi r^2")); h.pir2 = dp;
    }
    TRY(upload(c, &ip, mt, "mat")); h.mat = ip;
    TRY(upload(c, &ip, constrained, "constrained")); h.constrained = ip;
    h.n_groups = g->n_groups > 1 ? g->n_groups : 0;
    if (h.n_groups) {
        const int S = h.n_groups;
        std::vector<int> grp(g->group, g->group + B);
        TRY(upload(c, &ip, grp, "subelement groups")); h.group = ip;
        for (int k = 0; k < kGroupMax; ++k) h.gwt[k] = 0.0;
        for (int k = 0; k < B; ++k) h.gwt[grp[k]] += 1.0 / B;
        TRY(dalloc(c, &h.Itr, N, "transport part"));
        CK(cudaMemsetAsync(h.Itr, 0, N * sizeof(double), c->stream), "memset");
        TRY(dalloc(c, &h.xI, N, "transport rate"));
        TRY(dalloc(c, &h.zgrp, (size_t)N * S, "subelement projections"));
        TRY(dalloc(c, &h.ugrp, (size_t)W * S, "subelement voltages"));
    }
    TRY(upload(c, &ip, block_type, "block_type")); h.block_type = ip;

    // thermal / stencil tables
    if (sol) {
        TRY(upload(c, &ip, elem_grid, "elem_grid")); h.elem_grid = ip;
        TRY(upload(c, &ip, grid_elem, "grid_elem")); h.grid_elem = ip;
        std::vector<int> j0r, j0z;
        std::vector<double> wr, wz;
        stencil_axis(r_axis, j0r, wr);
        stencil_axis(z_axis, j0z, wz);
        TRY(upload(c, &ip, j0r, "sr_j0")); h.sr_j0 = ip;
        TRY(upload(c, &ip, j0z, "sz_j0")); h.sz_j0 = ip;
        TRY(upload(c, &dp, wr, "sr_w")); h.sr_w = dp;
        TRY(upload(c, &dp, wz, "sz_w")); h.sz_w = dp;
        // per element: the elements of its three stencil cells along r and along
        // z, with the cell's column / row in the fourth slot (a tap outside the
        // grid, whose weight is zero, names the element itself)
        std::vector<int4> tr(N), tz(N);
        for (int e = 0; e < N; ++e) {
            const int gg = elem_grid[e], iz = gg / Gr, ir = gg - iz * Gr;
            int t[6];
            for (int k = 0; k < 3; ++k) {
                const int jr = j0r[ir] + k, jz = j0z[iz] + k;
                t[k] = jr < Gr ? grid_elem[(size_t)iz * Gr + jr] : e;
                t[3 + k] = jz < Gz ? grid_elem[(size_t)jz * Gr + ir] : e;
            }
            tr[e] = make_int4(t[0], t[1], t[2], ir);
            tz[e] = make_int4(t[3], t[4], t[5], iz);
        }
        int4* tp;
        TRY(upload(c, &tp, tr, "stencil taps (r)")); h.tap_r = tp;
        TRY(upload(c, &tp, tz, "stencil taps (z)")); h.tap_z = tp;
        double T3 = 4.0 * m->T_ref * m->T_ref * m->T_ref;
        double Kin = m->kappa_cu / T3;
        double Kgap = gap > 0.0 ? hel / (hel / m->kappa_cu + gap / m->kappa_ep) / T3 : Kin;
        c->Kr_host.assign(Gr > 1 ? Gr - 1 : 0, Kin);
        c->Kz_host.assign(Gz > 1 ? Gz - 1 : 0, Kin);
        for (int i = 0; i + 1 < Gr; ++i)
            if ((i + 1) % n == 0) c->Kr_host[i] = Kgap;
        for (int j = 0; j + 1 < Gz; ++j)
            if ((j + 1) % n == 0) c->Kz_host[j] = Kgap;
        TRY(upload(c, &dp, c->Kr_host, "Kr")); h.Kr = dp;
        TRY(upload(c, &dp, c->Kz_host, "Kz")); h.Kz = dp;
        std::vector<int> nb((size_t)Gr * Gz);
        for (int j = 0; j < Gz; ++j)
            for (int i = 0; i < Gr; ++i)
                nb[(size_t)j * Gr + i] = (i == 0) + (i == Gr - 1) + (j == 0) + (j == Gz - 1);
        TRY(upload(c, &ip, nb, "nborder")); h.nborder = ip;
        h.Ccell = m->rho_m * m->c0 * hel * hel / 4.0;
        h.inv_Ccell = 1.0 / h.Ccell;
        h.helem = hel;
        h.src_k = 4.0 / (m->rho_m * m->c0);
        h.inv_Tref = 1.0 / m->T_ref;
        h.inv_h2 = 1.0 / (hel * hel);
        double* t6;
        TRY(dalloc(c, &t6, 3 * (size_t)Gr + 3 * (size_t)Gz, "thomas"));
        h.thr_a = t6; h.thr_inv = t6 + Gr; h.thr_c = t6 + 2 * Gr;
        h.thz_a = t6 + 3 * Gr; h.thz_inv = t6 + 3 * Gr + Gz; h.thz_c = t6 + 3 * Gr + 2 * Gz;
        std::vector<double> u0((size_t)Gr * Gz, m->T_bath * m->T_bath * m->T_bath * m->T_bath);
        TRY(upload(c, &h.uT, u0, "uT"));
        TRY(dalloc(c, &h.ustar, (size_t)Gr * Gz, "ustar"));
        TRY(dalloc(c, &h.src, (size_t)Gr * Gz, "src"));
        TRY(dalloc(c, &h.qgrid, (size_t)Gr * Gz, "qgrid"));
        TRY(dalloc(c, &h.partT, (size_t)Gr, "partT"));
    }

    // state and work vectors (ld long, zero padded, for the operator input)
    size_t ld = (size_t)h.ld;
    TRY(dalloc(c, &h.I, N, "I"));
    TRY(dalloc(c, &h.Phi, N, "Phi"));
    TRY(dalloc(c, &h.x, ld, "x"));
    TRY(dalloc(c, &h.xprev, N, "previous Idot"));
    TRY(dalloc(c, &h.xprev2, N, "Idot before the previous"));
    h.extrap = 1;
    h.rec_x = h.rec_res = h.rec_uw = h.rec_u = nullptr;
    h.rec_step0 = 0;
    h.rec_mode = 0;
    TRY(dalloc(c, &h.res, N, "res"));
    TRY(dalloc(c, &h.zv, N, "z"));
    TRY(dalloc(c, &h.dv, ld, "d"));
    TRY(dalloc(c, &h.qv, N, "q"));
    TRY(dalloc(c, &h.qn, N, "near part of q"));
    TRY(dalloc(c, &h.R, N, "R"));
    TRY(dalloc(c, &h.G, N, "G"));
    TRY(dalloc(c, &h.pf, ld, "pf"));
    TRY(dalloc(c, &h.L, (size_t)W * B * B, "L"));
    if (B <= kMedMax) TRY(dalloc(c, &h.Lf, (size_t)W * B * B, "preconditioner"));
    TRY(dalloc(c, &h.y1, (size_t)W * B, "y1"));
    TRY(dalloc(c, &h.sigma, W, "sigma"));
    TRY(dalloc(c, &h.isigma, W, "1 / sigma"));
    TRY(dalloc(c, &h.cw, W, "cw"));
    TRY(dalloc(c, &h.uw, W, "uw"));
    // 8 rows of W per-block partials; row 7 also takes the step end's 6
    // partials per CTA, so it is at least 6 kStepEndCtas long
    TRY(dalloc(c, &h.parts, 7 * (size_t)W + std::max<size_t>(W, 6 * kStepEndCtas), "parts"));
    TRY(dalloc(c, &h.first_jump, W, "first_jump"));
    TRY(dalloc(c, &h.first_quench, W, "first_quench"));
    CK(cudaMemsetAsync(h.first_jump, 0xff, W * sizeof(long long), c->stream), "memset");
    CK(cudaMemsetAsync(h.first_quench, 0xff, W * sizeof(long long), c->stream), "memset");
    TRY(dalloc(c, &h.wstat, 6 * (size_t)W, "wire statistics"));
    TRY(dalloc(c, &h.first_rise, W, "first_rise"));
    TRY(reset_wire_stats(c, false));
    h.acc_on = 1;
    TRY(dalloc(c, &h.diag, (size_t)h.diag_cap * COIL_DIAG_WIDTH, "diag"));
    TRY(dalloc(c, &h.sc, 1, "scalars"));
    TRY(dalloc(c, &h.ticket, 5, "arrival counters"));
    TRY(dalloc(c, &c->readbuf, 5 * (size_t)N + kMomentBlocks, "read buffer"));

    // operator: table of distinct entries, dense far part, FP64 near blocks
    size_t esz = o->precision == PREC_FP64 ? 8 : (o->precision == PREC_FP32 ? 4 : 2);
    const bool toep = o->format == COIL_FORMAT_TOEPLITZ;
    const bool tcf = o->format == COIL_FORMAT_TOEPLITZ_TC;
    h.op_format = toep ? 1 : (tcf ? 2 : 0);
    h.C = C;
    h.NT = NT;
    const size_t tab_entries = (size_t)C * C * (2 * (size_t)NT - 1);
    TcShape tsh{};
    if (tcf && !tc_shape(C, NT, c->n_sm, &tsh))
        return fail(c, COIL_ERR_INVALID, "coil shape not supported by the tensor-core Toeplitz format");
    const size_t op_alloc = toep ? tab_entries * sizeof(float)
                                 : (tcf ? tc_table_halves(tsh) * sizeof(__half) : (size_t)N * ld * esz);
    void* M = nullptr;
    {
        cudaError_t e = cudaMalloc(&M, op_alloc);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, COIL_ERR_OOM, "device allocation of the far operator failed (" +
                                             std::to_string(op_alloc) + " bytes)");
        }
        c->allocs.push_back(M);
        c->bytes += op_alloc;
        c->op_bytes = op_alloc;
    }
    if (toep) {
        TRY(dalloc(c, &h.tpart, toeplitz_part_floats(C, NT), "Toeplitz partial sums"));
        TRY(dalloc(c, &h.pT, N, "transposed operator input"));
    }
    if (tcf) {
        c->tc = new (std::nothrow) TcPlan();
        if (!c->tc) return fail(c, COIL_ERR_OOM, "host allocation of the tensor-core plan failed");
        TcPlan& P = *c->tc;
        P.sh = tsh;
        P.smem = tc_smem_bytes(tsh);
        P.t16 = static_cast<__half*>(M);
        TRY(dalloc(c, &P.p16, 2 * (size_t)tsh.Cp * NT, "split operator input"));
        TRY(tc_plan_schedule(c, tsh));
        TRY(dalloc(c, &P.pexp, (size_t)NT, "input scale exponents"));
        // the near kernels of small and medium wires sum the partial tiles themselves
        P.fused = B <= kSegMax || (B <= kMedMax && h.n_groups == 0);
        h.tc_part = P.part;
        h.tc_pexp = P.pexp;
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0), "event");
    CK(cudaEventCreate(&e1), "event");
    CK(cudaEventRecord(e0, c->stream), "event");
    double glx[4], glw[4];
    double s65 = sqrt(6.0 / 5.0);
    double xa = sqrt(3.0 / 7.0 - 2.0 / 7.0 * s65), xb = sqrt(3.0 / 7.0 + 2.0 / 7.0 * s65);
    double wa = (18.0 + sqrt(30.0)) / 36.0, wb = (18.0 - sqrt(30.0)) / 36.0;
    glx[0] = -xb; glx[1] = -xa; glx[2] = xa; glx[3] = xb;
    glw[0] = wb; glw[1] = wa; glw[2] = wa; glw[3] = wb;
    CK(upload_gl_rule(glx, glw), "gl rule");
    std::vector<double> rc(r.begin(), r.begin() + C), zc(z.begin(), z.begin() + C), hc(hh.begin(), hh.begin() + C);
    double *drc, *dzc, *dhc, *tab;
    TRY(upload(c, &drc, rc, "rc"));
    TRY(upload(c, &dzc, zc, "zc"));
    TRY(upload(c, &dhc, hc, "hc"));
    size_t tab_n = (size_t)C * C * (2 * (size_t)NT - 1);
    TRY(dalloc(c, &tab, tab_n, "operator table"));
    CK(launch_table(drc, dzc, dhc, C, NT, pitch_t, tab, c->stream), "table");
    if (toep) {
        h.tab32 = static_cast<const float*>(M);
        h.Mfar = nullptr;
        CK(launch_toeplitz_table(tab, C, NT, B, static_cast<float*>(M), c->stream), "Toeplitz table");
    } else if (tcf) {
        h.Mfar = nullptr;
        double* scratch;
        TRY(dalloc(c, &scratch, 1024, "scratch"));
        CK(tc_build_table(c->tc, tab, B, scratch, c->stream), "tensor-core Toeplitz table");
        h.tc_exT = c->tc->exT;
    } else {
        h.Mfar = M;
        CK(launch_expand(tab, C, NT, B, N, h.ld, o->precision, M, c->stream), "expand");
    }
    double* nearp;
    float* nearfp = nullptr;
    TRY(dalloc(c, &nearp, (size_t)n_types * B * B, "near blocks"));
    if (B <= kMedMax) TRY(dalloc(c, &nearfp, (size_t)n_types * B * B, "near blocks (FP32)"));
    CK(launch_near_blocks(tab, C, NT, B, n_types, nearp, nearfp, c->stream), "near blocks");
    h.near = nearp;
    h.nearf = nearfp;
    CK(cudaEventRecord(e1, c->stream), "event");
    CK(cudaStreamSynchronize(c->stream), "assembly");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    c->setup_ms = ms;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    // the table and channel arrays are no longer needed
    for (void* p : {(void*)tab, (void*)drc, (void*)dzc, (void*)dhc}) {
        for (size_t i = 0; i < c->allocs.size(); ++i)
            if (c->allocs[i] == p) { c->allocs.erase(c->allocs.begin() + i); break; }
        cudaFree(p);
    }
    c->bytes -= tab_n * sizeof(double) + 3 * (size_t)C * sizeof(double);

    CK(cudaMalloc(&c->d, sizeof(CoilDev)), "descriptor");
    CK(cudaHostAlloc(&c->pinned, sizeof(Scalars), cudaHostAllocDefault), "pinned scalars");
    memset(c->pinned, 0, sizeof(Scalars));
    CK(cudaMemcpyAsync(c->d, &h, sizeof(CoilDev), cudaMemcpyHostToDevice, c->stream), "descriptor");
    if (c->tc) {
        c->tc->d = c->d;
        const char* why = "";
        if (tc_encode_maps(c->tc, &why) != cudaSuccess) {
            cudaGetLastError();
            return fail(c, COIL_ERR_CUDA, why);
        }
        CK(cudaStreamSynchronize(c->stream), "create");
        TRY(tc_autotune(c, false));
    }
    CK(cudaStreamSynchronize(c->stream), "create");
    return COIL_OK;
}

// Per-wire statistics back to their empty values (heat and maxima 0, onset
// heat -1, first_rise -1); with onsets also first_jump and first_quench.
coil_status reset_wire_stats(coil_t* c, bool onsets) {
    const CoilDev& h = c->h;
    const size_t W = h.W;
    std::vector<double> init(6 * W, 0.0);
    std::fill(init.begin() + 3 * W, init.end(), -1.0);
    CK(cudaMemcpyAsync(h.wstat, init.data(), init.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream),
       "wire statistics");
    CK(cudaMemsetAsync(h.first_rise, 0xff, W * sizeof(long long), c->stream), "memset");
    if (onsets) {
        CK(cudaMemsetAsync(h.first_jump, 0xff, W * sizeof(long long), c->stream), "memset");
        CK(cudaMemsetAsync(h.first_quench, 0xff, W * sizeof(long long), c->stream), "memset");
    }
    CK(cudaStreamSynchronize(c->stream), "wire statistics");
    return COIL_OK;
}

coil_status sync_descriptor(coil_t* c) {
    CK(cudaMemcpyAsync(c->d, &c->h, sizeof(CoilDev), cudaMemcpyHostToDevice, c->stream), "descriptor");
    return COIL_OK;
}

coil_status set_drive(coil_t* c, const coil_drive* dr) {
    if (!dr || !(dr->dt > 0.0) || !is_fin(dr->dt) || !is_fin(dr->ramp_rate) || !is_fin(dr->I_max) ||
        !is_fin(dr->Ba_rate) || !is_fin(dr->Ba_max))
        return fail(c, COIL_ERR_INVALID, "drive needs a finite dt > 0 and finite rates");
    if (dr->Ba_waveform < 0 || dr->Ba_waveform > 2) return fail(c, COIL_ERR_INVALID, "unknown Ba_waveform");
    if (dr->Ba_waveform == 2 && dr->Ba_rate != 0.0 && !(dr->Ba_max > 0.0))
        return fail(c, COIL_ERR_INVALID, "triangle waveform needs Ba_max > 0");
    CoilDev& h = c->h;
    h.dt = dr->dt; h.ramp = dr->ramp_rate; h.Imax = dr->I_max;
    h.inv_dt = dr->dt > 0.0 ? 1.0 / dr->dt : 0.0;
    h.Ba_rate = dr->Ba_rate; h.Ba_max = dr->Ba_max; h.Ba_wf = dr->Ba_waveform;
    if (h.has_grid && c->thomas_dt != dr->dt) {
        std::vector<double> lo, inv, cp, lz, iz, cz;
        thomas_factors(c->Kr_host, 0.5 * dr->dt, h.Ccell, lo, inv, cp);
        thomas_factors(c->Kz_host, 0.5 * dr->dt, h.Ccell, lz, iz, cz);
        std::vector<double> all;
        all.insert(all.end(), lo.begin(), lo.end());
        all.insert(all.end(), inv.begin(), inv.end());
        all.insert(all.end(), cp.begin(), cp.end());
        all.insert(all.end(), lz.begin(), lz.end());
        all.insert(all.end(), iz.begin(), iz.end());
        all.insert(all.end(), cz.begin(), cz.end());
        CK(cudaMemcpyAsync((void*)h.thr_a, all.data(), all.size() * sizeof(double), cudaMemcpyHostToDevice,
                           c->stream), "thomas");
        CK(cudaStreamSynchronize(c->stream), "thomas");
        c->thomas_dt = dr->dt;
    }
    c->drive = *dr;
    c->has_drive = true;
    return sync_descriptor(c);
}

coil_status read_scalars(coil_t* c) {
    CK(cudaMemcpyAsync(c->pinned, c->h.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream), "scalars");
    CK(cudaStreamSynchronize(c->stream), "step");
    return COIL_OK;
}

size_t block_smem(const CoilDev& h) {
    const size_t S = h.n_groups;     // subelement scratch of the factor kernel
    return ((size_t)h.B * h.B + 2 * (size_t)h.B + (size_t)h.B * S + S * S) * sizeof(double);
}

// Launch geometry of one step for one coil or a batch (grid row y = coil).
struct Launch {
    const CoilDev* d = nullptr;
    // one coil of small blocks in the two-fill tensor-core form: the apply's
    // near warps form the near-block part of q (from x for the first apply of a
    // step, from d in the iterations) into qn, which the near kernel reads
    bool near_in_apply = false;
    const double *near_x = nullptr, *near_d = nullptr;
    double* near_q = nullptr;
    std::vector<const TcPlan*> tc;   // format 2: one plan per coil
    int n = 1;
    int prec = 0;
    int maxW = 0, maxN = 0, maxGr = 0, maxGz = 0;
    bool thermal = false;
    size_t smem = 0;
    cudaStream_t s = nullptr;
    int n_sm = 148;
    int format = 0;
    int maxC = 0, maxNT = 0;
    bool seg = false, big = false;   // coils with blocks of <= kSegMax / more elements present
    bool med = false, chol = false;  // of the latter: the FP32-inverse kernels (<= kMedMax, no
                                     // subelements) / the Cholesky ones
    bool groups = false;             // coils with subelements present
    bool need_q = false;             // the far apply must leave its result in q (no fused consumer)
    bool dir = false;                // format 2: the apply forms the PCG direction first
    // format 2 batches: side streams the coils' applies are spread over (fork
    // and join events: aux_ev[0..n_aux) per stream, aux_ev[n_aux] the fork)
    const cudaStream_t* aux = nullptr;
    const cudaEvent_t* aux_ev = nullptr;
    int n_aux = 0;
    // a graph-launched step's PCG iteration: (fuse_cond) the update kernel
    // sets the loop's condition
    bool fuse_cond = false;
    cudaGraphConditionalHandle cond = 0;
    // format 2 batches: every coil's apply in one launch of each kernel
    const TcBatch* tcb = nullptr;
};

Launch single_launch(coil_t* c) {
    Launch L;
    const CoilDev& h = c->h;
    L.d = c->d;
    L.n = 1;
    L.prec = h.precision;
    L.maxW = h.W;
    L.maxN = h.N;
    L.maxGr = h.Gr;
    L.maxGz = h.Gz;
    L.thermal = h.thermal != 0;
    L.smem = block_smem(h);
    L.s = c->stream;
    L.n_sm = c->n_sm;
    L.format = h.op_format;
    L.maxC = h.C;
    L.maxNT = h.NT;
    L.seg = h.B <= kSegMax;
    L.big = !L.seg;
    L.med = L.big && h.B <= kMedMax && h.n_groups == 0;
    L.chol = L.big && !L.med;
    L.groups = h.n_groups != 0;
    if (c->tc) L.tc.push_back(c->tc);
    L.near_in_apply = L.format == 2 && c->tc && c->tc->sh.mode == 0 && L.seg;
    L.near_x = h.x;
    L.near_d = h.dv;
    L.near_q = h.qn;
    return L;
}

// The far-operator apply of either storage format.
cudaError_t launch_far(const Launch& L, int which) {
    if (L.format == 1) return launch_toeplitz(L.d, L.n, L.maxC, L.maxNT, L.maxN, L.n_sm, L.s);
    if (L.format == 2) {
        if (L.tcb && L.tc.size() > 1) return launch_tc_batch(*L.tcb, L.s, L.need_q, L.dir);
        if (L.n_aux > 0 && L.tc.size() > 1) {
            // a batch: the coils' applies are independent, so they run side by
            // side on the side streams (one SM per CTA each: a small coil's
            // apply alone leaves most of the GPU idle)
            cudaError_t e = cudaEventRecord(L.aux_ev[L.n_aux], L.s);
            for (int a = 0; a < L.n_aux && e == cudaSuccess; ++a) e = cudaStreamWaitEvent(L.aux[a], L.aux_ev[L.n_aux], 0);
            for (size_t i = 0; i < L.tc.size() && e == cudaSuccess; ++i)
                e = launch_toeplitz_tc(*L.tc[i], L.aux[i % L.n_aux], L.need_q || !L.tc[i]->fused, L.dir);
            for (int a = 0; a < L.n_aux && e == cudaSuccess; ++a) {
                e = cudaEventRecord(L.aux_ev[a], L.aux[a]);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(L.s, L.aux_ev[a], 0);
            }
            return e;
        }
        for (const TcPlan* P : L.tc) {
            const bool nia = L.near_in_apply && L.tc.size() == 1;
            cudaError_t e = launch_toeplitz_tc(*P, L.s, L.need_q || !P->fused, L.dir,
                                               nia ? (which == 0 ? L.near_x : L.near_d) : nullptr,
                                               nia ? L.near_q : nullptr);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    return launch_gemv(L.d, L.n, L.prec, L.maxN, which, L.n_sm, L.s);
}

// Dense-operator launch, bracketed by an event pair when profiling.
coil_status gemv(coil_t* c, const Launch& L, int which) {
    if (c->profile && L.format == 2 && L.tc.size() == 1 && L.n_aux == 0) {
        // the tensor-core form: the events bracket its product kernel alone
        // (the input split is a kernel of its own)
        if (c->ev_used * 2 + 2 > c->ev_pool.size()) {
            for (int k = 0; k < 2; ++k) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e), "event");
                c->ev_pool.push_back(e);
            }
        }
        const TcPlan& P = *L.tc[0];
        CK(launch_tc_split(P, L.s, L.dir), "operator apply");
        CK(cudaEventRecord(c->ev_pool[2 * c->ev_used], L.s), "event");
        CK(launch_tc_apply(P, L.s, L.need_q || !P.fused, L.near_in_apply ? (which == 0 ? L.near_x : L.near_d) : nullptr,
                           L.near_in_apply ? L.near_q : nullptr),
           "operator apply");
        CK(cudaEventRecord(c->ev_pool[2 * c->ev_used + 1], L.s), "event");
        c->ev_used += 1;
        c->op_launches += 1;
        c->launches += 1;
        return COIL_OK;
    }
    if (c->profile) {
        if (c->ev_used * 2 + 2 > c->ev_pool.size()) {
            for (int k = 0; k < 2; ++k) {
                cudaEvent_t e;
                CK(cudaEventCreate(&e), "event");
                c->ev_pool.push_back(e);
            }
        }
        CK(cudaEventRecord(c->ev_pool[2 * c->ev_used], L.s), "event");
    }
    CK(launch_far(L, which), "operator apply");
    if (c->profile) {
        CK(cudaEventRecord(c->ev_pool[2 * c->ev_used + 1], L.s), "event");
        c->ev_used += 1;
    }
    c->op_launches += 1;
    c->launches += 1;
    return COIL_OK;
}

// Sum the recorded operator intervals (call after a stream synchronize).
void harvest_events(coil_t* c) {
    for (size_t i = 0; i < c->ev_used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev_pool[2 * i], c->ev_pool[2 * i + 1]) == cudaSuccess) c->op_ms += ms;
    }
    c->ev_used = 0;
}

dim3 warp_grid(const Launch& L) { return dim3((unsigned)((L.maxW + 7) / 8), L.n); }

// Near-block product, initial residual and PCG update: one warp per wire for
// blocks of more than kSegMax elements, shared warps (at least two wires per
// warp) for smaller ones; a batch with both kinds launches both kernels, each
// skipping the other kind's coils.  Return the number of launches.
int launch_near(const Launch& L, int which, bool skip_seg = false) {
    if (L.chol) k_near<<<warp_grid(L), 256, 0, L.s>>>(L.d, which);
    // tensor-core format: small- and medium-block coils take the far part from
    // the partial tiles
    const int far_tiles = L.format == 2 && !L.need_q;
    if (L.med) k_near_med<<<dim3(L.maxW, L.n), kMedMax, 0, L.s>>>(L.d, which, far_tiles, which == 1);
    if (L.seg && !skip_seg)
        k_near_seg<<<dim3((unsigned)((L.maxW + 15) / 16), L.n), 256, 0, L.s>>>(L.d, which, far_tiles, which == 1,
                                                                              (int)L.near_in_apply);
    return (int)L.chol + (int)L.med + (int)(L.seg && !skip_seg);
}
// fuse: the small-block coils' init kernel reduces r^T z itself (last CTA).
// fuse_near: it also forms their A x0 (launch_near then skips k_near_seg).
int launch_init(const Launch& L, bool fuse, bool fuse_near = false) {
    if (L.chol) k_init<<<dim3(L.maxW, L.n), 32, L.smem, L.s>>>(L.d);
    if (L.med) k_init_med<<<dim3(L.maxW, L.n), kMedMax, 0, L.s>>>(L.d, (int)fuse);
    const int far_tiles = L.format == 2 && !L.need_q;
    if (L.seg)
        k_init_seg<<<dim3((unsigned)((L.maxW + 2 * kSegWarps - 1) / (2 * kSegWarps)), L.n), 32 * kSegWarps, 0, L.s>>>(
            L.d, (int)fuse, (int)fuse_near, far_tiles, (int)L.near_in_apply);
    return (int)L.chol + (int)L.med + (int)L.seg;
}
int launch_pointwise(const Launch& L) {
    if (L.big) k_pointwise<<<warp_grid(L), 256, 0, L.s>>>(L.d);
    if (L.seg) k_pointwise_seg<<<dim3((unsigned)((L.maxW + 15) / 16), L.n), 256, 0, L.s>>>(L.d);
    return (int)L.big + (int)L.seg;
}
// fuse: the small-block coils without subelements reduce the stopping scale
// in their factor kernel (last CTA).
int launch_factor(const Launch& L, bool fuse) {
    if (L.chol) k_factor<<<dim3(L.maxW, L.n), 32, L.smem, L.s>>>(L.d);
    if (L.med) k_factor_med<<<dim3(L.maxW, L.n), kMedFactorThreads, 0, L.s>>>(L.d, (int)fuse);
    if (L.seg) {
        const dim3 grid((unsigned)((L.maxW + 2 * kSegWarps - 1) / (2 * kSegWarps)), L.n);
        k_factor_seg<<<grid, 32 * kSegWarps, 0, L.s>>>(L.d, (int)fuse);
        if (L.groups) k_factor_seg_groups<<<grid, 32 * kSegWarps, 0, L.s>>>(L.d);
        return (int)L.chol + (int)L.med + 1 + (int)L.groups;
    }
    return (int)L.chol + (int)L.med + (int)L.seg;
}
int launch_update(const Launch& L) {
    if (L.chol) k_update<<<dim3(L.maxW, L.n), 32, L.smem, L.s>>>(L.d);
    if (L.med) k_update_med<<<dim3(L.maxW, L.n), kMedMax, 0, L.s>>>(L.d, 1, L.cond, (int)L.fuse_cond);
    if (L.seg)
        k_update_seg<<<dim3((unsigned)((L.maxW + 2 * kSegWarps - 1) / (2 * kSegWarps)), L.n), 32 * kSegWarps, 0, L.s>>>(
            L.d, 1, L.cond, (int)L.fuse_cond);
    return (int)L.chol + (int)L.med + (int)L.seg;
}

// The solve's first two reductions for the coils whose kernels do not fuse
// them (the Cholesky path's; subelement coils' for the scale).
int scale_reduce(const Launch& L) {
    if (!L.chol && !L.groups) return 0;
    k_reduce<<<L.n, kRedThreads, 0, L.s>>>(L.d, 0, 2);
    return 1;
}
int init_reduce(const Launch& L) {
    if (!L.chol) return 0;
    k_reduce<<<L.n, kRedThreads, 0, L.s>>>(L.d, 1, 1);
    return 1;
}

// Pointwise, factorisation, right-hand-side norm, initial residual.
coil_status step_prologue(coil_t* c, const Launch& L) {
    c->launches += launch_pointwise(L);
    c->launches += launch_factor(L, true);
    c->launches += scale_reduce(L);
    TRY(gemv(c, L, 0));
    c->launches += launch_near(L, 0, true);
    c->launches += launch_init(L, true, true);
    c->launches += init_reduce(L);
    CK(cudaGetLastError(), "step launch");
    return COIL_OK;
}

// One projected-PCG iteration (kernels of converged coils return at once).
// The tensor-core format forms the direction d = -z + beta d inside the input
// split of the iteration that uses it (from the second iteration on).
coil_status step_iteration(coil_t* c, const Launch& L) {
    const bool fuse_dir = L.format == 2;
    if (fuse_dir) {
        Launch Ld = L;
        Ld.dir = true;
        TRY(gemv(c, Ld, 1));
    } else {
        TRY(gemv(c, L, 1));
    }
    // small- and medium-block coils reduce alpha and beta in the last CTA of their kernels
    c->launches += launch_near(L, 1);
    if (L.chol) k_reduce<<<L.n, kRedThreads, 0, L.s>>>(L.d, 2, 1);
    c->launches += launch_update(L);
    if (L.chol) k_reduce<<<L.n, kRedThreads, 0, L.s>>>(L.d, 3, 1);
    if (!fuse_dir) {
        unsigned eb = (unsigned)((L.maxN + 255) / 256);
        if (eb > (unsigned)L.n_sm * 16) eb = L.n_sm * 16;
        k_direction<<<dim3(eb, L.n), 256, 0, L.s>>>(L.d);
        c->launches += 1;
    }
    c->launches += 2 * (int)L.chol;
    CK(cudaGetLastError(), "iteration launch");
    return COIL_OK;
}

// Current/flux update, heat step, diagnostics (coils whose solve failed skip it).
coil_status step_epilogue(coil_t* c, const Launch& L) {
    if (L.big || L.groups) {
        k_finalize<<<warp_grid(L), 256, 0, L.s>>>(L.d);
        c->launches += 1;
    }
    if (L.seg) {
        k_finalize_seg<<<dim3((unsigned)((L.maxW + 15) / 16), L.n), 256, 0, L.s>>>(L.d);
        c->launches += 1;
    }
    if (L.thermal) {
        k_adi_r<<<dim3(L.maxGz, L.n), kAdiThreads, adi_smem_bytes(L.maxGr), L.s>>>(L.d);
        k_adi_z<<<dim3(L.maxGr, L.n), kAdiThreads, adi_smem_bytes(L.maxGz), L.s>>>(L.d);
        c->launches += 2;
    }
    k_step_end<<<dim3(kStepEndCtas, L.n), kStepEndThreads, 0, L.s>>>(L.d);
    c->launches += 1;
    CK(cudaGetLastError(), "step end launch");
    return COIL_OK;
}

// Capture one step as a graph: the prologue, a while node whose body is one
// PCG iteration whose update kernel's last CTA (or, for coils with blocks of
// more than 16 elements, k_loop_cond) sets the loop's condition (the device
// decides when to stop), the epilogue (its kernels skip a failed step) and the
// copy of the scalars to the pinned mirror; the adjoint's transposed solve the
// same way with its own prologue and no epilogue.  One launch and one
// synchronization per step instead of
// ~5 launches per iteration and a host check per chunk of iterations.
coil_status adjoint_prologue(coil_t* c, const Launch& L);

// kind 0: the forward step (step_prologue, loop, step_epilogue, scalars); kind
// 1: the adjoint's transposed solve (adjoint_prologue, loop, scalars); kind 2:
// a batched step (L over the batch's coils, bg its descriptors and status:
// pass counter reset, step_prologue, loop with k_batch_cond, step_epilogue,
// status gathered and copied to bg->hstat).
coil_status build_step_graph(coil_t* c, int kind = 0, const Launch* Lbatch = nullptr, BatchGraph* bg = nullptr,
                             int maxit = 0) {
    cudaStream_t s = c->stream;
    Launch L = kind == 2 ? *Lbatch : single_launch(c);
    const int n = L.n;
    // the side streams of a batch's tensor-core applies join the loop body's
    // capture only: the prologue's apply runs its coils one after another
    Launch Lp = L;
    Lp.aux = nullptr;
    Lp.aux_ev = nullptr;
    Lp.n_aux = 0;
    int* dstat = kind == 2 ? reinterpret_cast<int*>(bg->dd + n) : nullptr;
    if (!c->body_stream) CK(cudaStreamCreateWithFlags(&c->body_stream, cudaStreamNonBlocking), "graph stream");
    const long long l0 = c->launches, op0 = c->op_launches;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, "step capture");
    if (kind == 2) e = cudaMemsetAsync(dstat + 3 * n, 0, sizeof(int), s);   // the batch's pass counter
    coil_status st = kind == 1 ? adjoint_prologue(c, Lp) : step_prologue(c, Lp);
    cudaStreamCaptureStatus cs;
    cudaGraph_t cg = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    cudaGraphConditionalHandle hnd = 0;
    cudaGraphNodeParams np = {};
    cudaGraphNode_t cnode = nullptr;
    if (st == COIL_OK) e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, nullptr, &nd);
    if (st == COIL_OK && e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hnd, cg, 1, cudaGraphCondAssignDefault);
    if (st == COIL_OK && e == cudaSuccess) {
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = hnd;
        np.conditional.type = cudaGraphCondTypeWhile;
        np.conditional.size = 1;
        e = cudaGraphAddNode(&cnode, cg, deps, nullptr, nd, &np);
    }
    if (st == COIL_OK && e == cudaSuccess)
        e = cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies);
    const long long l1 = c->launches;
    if (st == COIL_OK && e == cudaSuccess) {
        e = cudaStreamBeginCaptureToGraph(c->body_stream, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            Launch Lb = L;
            Lb.s = c->body_stream;
            Lb.cond = hnd;
            Lb.fuse_cond = kind != 2 && !L.chol;   // the shared-warp or medium-wire update kernel's last CTA
            st = step_iteration(c, Lb);
            if (kind == 2) {
                k_batch_cond<<<1, 128, 0, c->body_stream>>>(L.d, n, dstat + 3 * n, maxit, hnd);
                c->launches += 1;
            } else if (!Lb.fuse_cond) {
                k_loop_cond<<<1, 1, 0, c->body_stream>>>(c->d, hnd);
                c->launches += 1;
            }
            cudaGraph_t body = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(c->body_stream, &body);
            if (e == cudaSuccess) e = e2;
        }
    }
    const long long l2 = c->launches;
    if (st == COIL_OK && e == cudaSuccess && kind != 1) st = step_epilogue(c, Lp);
    if (st == COIL_OK && e == cudaSuccess && kind == 2) {
        k_gather_status<<<(n + 127) / 128, 128, 0, s>>>(L.d, n, dstat);
        c->launches += 1;
    }
    const long long l3 = c->launches;
    if (st == COIL_OK && e == cudaSuccess) {
        if (kind == 2)
            e = cudaMemcpyAsync(bg->hstat, dstat, (3 * n + 1) * sizeof(int), cudaMemcpyDeviceToHost, s);
        else
            e = cudaMemcpyAsync(c->pinned, c->h.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, s);
    }
    cudaError_t e3 = cudaStreamEndCapture(s, &g);
    if (e == cudaSuccess) e = e3;
    c->launches = l0;                                // counted per launch of the graph instead
    c->op_launches = op0;
    cudaGraphExec_t* exec = kind == 0 ? &c->step_exec : (kind == 1 ? &c->adj_exec : &bg->exec);
    if (st == COIL_OK && e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (st != COIL_OK) return st;
    if (e != cudaSuccess) {
        cudaGetLastError();
        *exec = nullptr;
        return cuda_fail(c, e, "step graph");
    }
    const int fixed = (int)((l1 - l0) + (l3 - l2)), per_pass = (int)(l2 - l1);
    if (kind == 0) { c->graph_fixed = fixed; c->graph_per_pass = per_pass; }
    else if (kind == 1) { c->adj_fixed = fixed; c->adj_per_pass = per_pass; }
    else { bg->fixed = fixed; bg->per_pass = per_pass; }
    return COIL_OK;
}

coil_status run_step(coil_t* c) {
    const CoilDev& h = c->h;
    if (!c->profile && !c->graph_failed) {
        if (!c->step_exec && build_step_graph(c) != COIL_OK) {
            c->graph_failed = true;                      // the same kernels, launched one by one
            c->err.clear();
        }
        if (c->step_exec) {
            CK(cudaGraphLaunch(c->step_exec, c->stream), "step graph launch");
            CK(cudaStreamSynchronize(c->stream), "step");
            const int passes = c->pinned->passes > 0 ? c->pinned->passes : 1;
            c->launches += c->graph_fixed + (long long)c->graph_per_pass * passes;
            c->op_launches += 1 + passes;
            int st = c->pinned->status;
            if (st == ST_KERNEL) return fail(c, COIL_ERR_CUDA, tc_timeout_text(c));
            if (!c->pinned->done || st == ST_NOT_CONVERGED)
                return fail(c, COIL_ERR_NOT_CONVERGED, "per-step solve did not converge within maxit iterations");
            if (st == ST_NONFINITE)
                return fail(c, COIL_ERR_NONFINITE, "non-finite value or non-positive pivot in the step solve");
            c->last_iters = c->pinned->iter > 0 ? c->pinned->iter : 1;
            c->pcg_iters += c->pinned->iter;
            c->steps += 1;
            c->t += h.dt;
            return COIL_OK;
        }
    }
    Launch L = single_launch(c);
    TRY(step_prologue(c, L));
    // PCG: enqueue the expected number of iterations, then one at a time
    // (profiling: one at a time throughout, so that no timed apply is one
    // enqueued after convergence, which returns at once)
    int chunk = !c->profile && c->last_iters > 1 ? c->last_iters : 1;
    int total = 0;
    for (;;) {
        for (int i = 0; i < chunk; ++i) TRY(step_iteration(c, L));
        total += chunk;
        TRY(read_scalars(c));
        if (c->pinned->done) break;
        if (total > h.maxit + 2) break;
        chunk = 1;
    }
    int st = c->pinned->status;
    if (st == ST_KERNEL) return fail(c, COIL_ERR_CUDA, tc_timeout_text(c));
    if (!c->pinned->done || st == ST_NOT_CONVERGED)
        return fail(c, COIL_ERR_NOT_CONVERGED, "per-step solve did not converge within maxit iterations");
    if (st == ST_NONFINITE)
        return fail(c, COIL_ERR_NONFINITE, "non-finite value or non-positive pivot in the step solve");
    c->last_iters = c->pinned->iter > 0 ? c->pinned->iter : 1;
    c->pcg_iters += c->pinned->iter;
    harvest_events(c);
    TRY(step_epilogue(c, L));
    c->steps += 1;
    c->t += h.dt;
    return COIL_OK;
}

// A replayed forward step of the adjoint's recomputation (rec_mode 2): the
// pointwise update and the factor (y = A_w^-1 1 and 1/sigma, which the
// finalisation reads) as in the step, then the recorded solution, residual
// and loop voltages in place of the solve, then the step's epilogue.
coil_status replay_kernels(coil_t* c, const Launch& L) {
    // no factorisation: the replay does not solve, and its finalisation takes
    // the recorded voltages in place of forming them from y and sigma
    c->launches += launch_pointwise(L);
    const unsigned nb = (unsigned)std::min<long long>(((long long)c->h.N + 255) / 256, 148LL * 8);
    k_replay_restore<<<dim3(nb, L.n), 256, 0, L.s>>>(L.d);
    c->launches += 1;
    CK(cudaGetLastError(), "replay launch");
    return step_epilogue(c, L);
}

coil_status run_replay_step(coil_t* c) {
    const CoilDev& h = c->h;
    if (!c->profile && !c->graph_failed && !c->replay_exec) {
        // one graph: the replay kernels and the scalars read back
        const long long l0 = c->launches;
        cudaGraph_t g = nullptr;
        coil_status st = COIL_ERR_CUDA;
        cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            st = replay_kernels(c, single_launch(c));
            if (st == COIL_OK)
                e = cudaMemcpyAsync(c->pinned, c->h.sc, sizeof(Scalars), cudaMemcpyDeviceToHost, c->stream);
            cudaError_t e2 = cudaStreamEndCapture(c->stream, &g);      // always ends the capture
            if (e == cudaSuccess) e = e2;
        }
        c->replay_fixed = (int)(c->launches - l0);
        c->launches = l0;
        if (st == COIL_OK && e == cudaSuccess) e = cudaGraphInstantiate(&c->replay_exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (st != COIL_OK || e != cudaSuccess) {
            cudaGetLastError();
            c->replay_exec = nullptr;
            c->graph_failed = true;                  // the same kernels, launched one by one
            c->err.clear();
        }
    }
    if (c->replay_exec) {
        CK(cudaGraphLaunch(c->replay_exec, c->stream), "replay graph launch");
        CK(cudaStreamSynchronize(c->stream), "replay");
        c->launches += c->replay_fixed;
    } else {
        TRY(replay_kernels(c, single_launch(c)));
        TRY(read_scalars(c));
    }
    const int st = c->pinned->status;
    if (st == ST_KERNEL) return fail(c, COIL_ERR_CUDA, tc_timeout_text(c));
    if (st != ST_OK) return fail(c, COIL_ERR_NONFINITE, "replayed step of the adjoint failed");
    c->steps += 1;
    c->t += h.dt;
    return COIL_OK;
}

// y = M p with FP64 near blocks (no dt G term): p -> x (and its FP32 copy),
// result in q.  Leaves x = 0 afterwards (cold warm start).
coil_status apply_plain(coil_t* c, const double* dev_p) {
    CoilDev& h = c->h;
    cudaStream_t s = c->stream;
    double dt_save = h.dt;
    h.dt = 0.0;
    TRY(sync_descriptor(c));
    CK(cudaMemcpyAsync(h.x, dev_p, h.N * sizeof(double), cudaMemcpyDeviceToDevice, s), "apply");
    CK(cudaMemsetAsync(&h.sc->done, 0, sizeof(int), s), "apply");
    k_to_float<<<(h.N + 255) / 256, 256, 0, s>>>(h.x, h.pf, h.N);
    CK(launch_far(single_launch(c), 0), "operator apply");
    launch_near(single_launch(c), 0);
    CK(cudaGetLastError(), "apply");
    h.dt = dt_save;
    TRY(sync_descriptor(c));
    if (h.op_format == 2) {
        TRY(read_scalars(c));
        if (c->pinned->status == ST_KERNEL) return fail(c, COIL_ERR_CUDA, tc_timeout_text(c));
    }
    return COIL_OK;
}

}  // namespace

namespace cq {
__global__ void k_to_float(const double* x, float* f, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) f[i] = (float)x[i];
}

// done, status, iter of every coil of a batch into one small array.
__global__ void k_gather_status(const CoilDev* __restrict__ cds, int n, int* out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const Scalars* sc = cds[i].sc;
        out[3 * i] = sc->done;
        out[3 * i + 1] = sc->status;
        out[3 * i + 2] = sc->iter;
    }
}

// Condition of a graph-launched batched step's PCG while loop: go on while
// any coil's solve is not done; past maxit + 2 passes the unfinished coils end
// as not converged, so the loop always terminates.  One CTA.
__global__ void k_batch_cond(const CoilDev* __restrict__ cds, int n, int* passes, int maxit,
                             cudaGraphConditionalHandle h) {
    __shared__ int p;
    if (threadIdx.x == 0) p = ++*passes;
    __syncthreads();
    int open = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        Scalars* sc = cds[i].sc;
        if (!sc->done) {
            if (p > maxit + 2) {
                sc->status = ST_NOT_CONVERGED;
                sc->done = 1;
            } else {
                open = 1;
            }
        }
    }
    open = __syncthreads_or(open);
    if (threadIdx.x == 0) cudaGraphSetConditional(h, open ? 1u : 0u);
}

// Moment sum(pi r^2 I) in two fixed-order passes: a grid-strided partial per
// block (the FP64 pipe of one SM alone takes ~0.2 ms at 96,000 elements), then
// one warp sums the partials.
__global__ void k_moment(const CoilDev* __restrict__ cds, double* part) {
    const CoilDev& c = *cds;
    __shared__ double sh[32];
    double m = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < c.N; e += gridDim.x * blockDim.x) {
        double r = c.r[e];
        m += kPi * r * r * c.I[e];
    }
    m = warp_sum(m);
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = m;
    __syncthreads();
    if (wid == 0) {
        m = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        m = warp_sum(m);
        if (lane == 0) part[blockIdx.x] = m;
    }
}

__global__ void k_moment_sum(const double* part, int n, double* out) {
    double m = 0.0;
    for (int k = threadIdx.x; k < n; k += 32) m += part[k];
    m = warp_sum(m);
    if (threadIdx.x == 0) *out = m;
}
}  // namespace cq

// ============================================================== C ABI

extern "C" {

coil_status coil_create(const coil_geometry* geom, const coil_material* mat, const coil_options* opt,
                        coil_t** out) {
    if (!out) return COIL_ERR_INVALID;
    *out = nullptr;
    coil_t* c = new (std::nothrow) coil();
    if (!c) return COIL_ERR_OOM;
    static std::atomic<long long> next_uid{1};
    c->uid = next_uid++;
    coil_status st = validate(geom, mat, opt, c);
    if (st == COIL_OK) {
        cudaError_t e = cudaSetDevice(opt->device);
        if (e != cudaSuccess) {
            st = cuda_fail(c, e, "cudaSetDevice");
        } else {
            c->device = opt->device;
            c->profile = opt->profile ? 1 : 0;
            cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, opt->device);
            if (opt->stream) {
                c->stream = (cudaStream_t)opt->stream;
            } else {
                e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
                if (e != cudaSuccess) st = cuda_fail(c, e, "stream");
                else c->own_stream = true;
            }
            if (st == COIL_OK) st = setup(c, geom, mat, opt);
        }
    }
    if (st != COIL_OK) {
        fprintf(stderr, "coil_create: %s\n", c->err.c_str());
        coil_destroy(c);
        return st;
    }
    *out = c;
    return COIL_OK;
}

coil_status coil_step(coil_t* c, long n_steps, const coil_drive* drive) {
    if (!c) return COIL_ERR_INVALID;
    if (n_steps < 0) return fail(c, COIL_ERR_INVALID, "n_steps must be >= 0");
    cudaSetDevice(c->device);
    TRY(set_drive(c, drive));
    if (c->tc && c->tc->in_batch) {
        // stepped alone again after batched steps: back to the autotuner's schedule
        TRY(tc_plan_schedule(c, c->tc->tuned_sh));
        c->tc->in_batch = false;
    }
    for (long k = 0; k < n_steps; ++k) TRY(run_step(c));
    CK(cudaStreamSynchronize(c->stream), "coil_step");
    return COIL_OK;
}

coil_status coil_batch_step(coil_t* const* coils, int n, long n_steps, const coil_drive* drives) {
    if (!coils || n < 1 || !drives || n_steps < 0) return COIL_ERR_INVALID;
    coil_t* c = coils[0];
    for (int i = 0; i < n; ++i) {
        if (!coils[i]) return COIL_ERR_INVALID;
        if (coils[i]->device != c->device || coils[i]->h.precision != c->h.precision ||
            coils[i]->h.op_format != c->h.op_format)
            return fail(c, COIL_ERR_INVALID, "batched coils must share device, precision and operator format");
        for (int j = 0; j < i; ++j)
            if (coils[j] == coils[i]) return fail(c, COIL_ERR_INVALID, "a coil appears twice in the batch");
    }
    cudaSetDevice(c->device);
    if (c->h.op_format == 2 && n > 1) {
        // batched tensor-core applies: each coil takes the two-fill schedule with
        // its step floor per CTA (not the autotuner's choice for running alone),
        // and the CTAs of all coils run in one launch
        bool replanned = false;
        for (int i = 0; i < n; ++i) {
            coil_t* ci = coils[i];
            if (!ci->tc || ci->tc->in_batch) continue;
            TcShape sb;
            if (!tc_shape(ci->tc->sh.C, ci->tc->sh.NT, ci->n_sm, &sb))
                return fail(c, COIL_ERR_INVALID, "coil shape not supported by the tensor-core Toeplitz format");
            TRY(tc_plan_schedule(ci, sb));
            ci->tc->in_batch = true;
            replanned = true;
        }
        std::vector<long long> ids(n);
        for (int i = 0; i < n; ++i) ids[i] = coils[i]->uid;
        if (replanned || !c->tcb || c->tcb_ids != ids) {
            // the schedules' buffers or the coil set changed: new arguments, new graph
            CK(cudaStreamSynchronize(c->stream), "batch applies");
            if (c->batch) {
                if (c->batch->exec) cudaGraphExecDestroy(c->batch->exec);
                cudaFree(c->batch->dd);
                cudaFreeHost(c->batch->hstat);
                delete c->batch;
                c->batch = nullptr;
            }
            if (!c->tcb) c->tcb = new TcBatch();
            std::vector<const TcPlan*> plans;
            for (int i = 0; i < n; ++i) plans.push_back(coils[i]->tc);
            CK(tc_batch_build(c->tcb, plans, c->stream), "batch applies");
            c->tcb_ids = ids;
        }
    }
    Launch L;
    L.n = n;
    L.prec = c->h.precision;
    L.s = c->stream;
    L.n_sm = c->n_sm;
    L.format = c->h.op_format;
    std::vector<CoilDev> hd(n);
    for (int i = 0; i < n; ++i) {
        coil_t* ci = coils[i];
        TRY(set_drive(ci, &drives[i]));
        CK(cudaStreamSynchronize(ci->stream), "batch descriptor");
        hd[i] = ci->h;
        L.maxW = std::max(L.maxW, ci->h.W);
        L.maxN = std::max(L.maxN, ci->h.N);
        L.maxGr = std::max(L.maxGr, ci->h.Gr);
        L.maxGz = std::max(L.maxGz, ci->h.Gz);
        L.thermal = L.thermal || ci->h.thermal;
        L.smem = std::max(L.smem, block_smem(ci->h));
        L.maxC = std::max(L.maxC, ci->h.C);
        L.maxNT = std::max(L.maxNT, ci->h.NT);
        L.seg = L.seg || ci->h.B <= kSegMax;
        L.big = L.big || ci->h.B > kSegMax;
        const bool med_i = ci->h.B > kSegMax && ci->h.B <= kMedMax && ci->h.n_groups == 0;
        L.med = L.med || med_i;
        L.chol = L.chol || (ci->h.B > kSegMax && !med_i);
        L.groups = L.groups || ci->h.n_groups != 0;
        if (ci->tc) L.tc.push_back(ci->tc);
    }
    if (L.format == 2 && n > 1 && c->tcb) {
        L.tcb = c->tcb;
    } else if (L.format == 2 && n > 1) {
        if (c->aux.empty()) {
            for (int a = 0; a < kAuxStreams; ++a) {
                cudaStream_t st;
                CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "batch streams");
                c->aux.push_back(st);
            }
            for (int a = 0; a <= kAuxStreams; ++a) {
                cudaEvent_t ev;
                CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "batch events");
                c->aux_ev.push_back(ev);
            }
        }
        L.aux = c->aux.data();
        L.aux_ev = c->aux_ev.data();
        L.n_aux = (int)c->aux.size();
    }
    int maxit = 0;
    for (int i = 0; i < n; ++i) maxit = std::max(maxit, coils[i]->h.maxit);
    // per coil after a step: counters on success, the first failure reported
    auto finish_step = [&](const int* hs) {
        coil_status first_err = COIL_OK;
        for (int i = 0; i < n; ++i) {
            coil_t* ci = coils[i];
            int done = hs[3 * i], st = hs[3 * i + 1], it = hs[3 * i + 2];
            if (done && st == ST_OK) {
                ci->steps += 1;
                ci->t += ci->h.dt;
                ci->last_iters = it > 0 ? it : 1;
                ci->pcg_iters += it;
            } else if (first_err == COIL_OK) {
                first_err = st == ST_KERNEL ? COIL_ERR_CUDA
                            : (!done || st == ST_NOT_CONVERGED) ? COIL_ERR_NOT_CONVERGED : COIL_ERR_NONFINITE;
                fail(ci, first_err, "batched step: this coil's solve failed; its state was kept");
            }
        }
        if (first_err != COIL_OK) fail(c, first_err, "batched step: at least one coil's solve failed");
        return first_err;
    };
    // graph-launched steps: the batch's step captured once (prologue, the PCG
    // loop over every coil until all are done, epilogue, status copy) and kept
    // by the first coil for later calls with the same coils
    if (!c->profile && !c->graph_failed) {
        std::vector<long long> ids(n);
        for (int i = 0; i < n; ++i) ids[i] = coils[i]->uid;
        if (c->batch && c->batch->ids != ids) {
            CK(cudaStreamSynchronize(L.s), "batch graph");
            if (c->batch->exec) cudaGraphExecDestroy(c->batch->exec);
            cudaFree(c->batch->dd);
            cudaFreeHost(c->batch->hstat);
            delete c->batch;
            c->batch = nullptr;
        }
        bool fresh = false;
        if (!c->batch) {
            BatchGraph* bg = new BatchGraph;
            bg->ids = ids;
            cudaError_t ea = cudaMalloc(&bg->dd, n * sizeof(CoilDev) + (3 * (size_t)n + 1) * sizeof(int));
            if (ea == cudaSuccess) ea = cudaMallocHost(&bg->hstat, (3 * (size_t)n + 1) * sizeof(int));
            if (ea == cudaSuccess)
                ea = cudaMemcpyAsync(bg->dd, hd.data(), n * sizeof(CoilDev), cudaMemcpyHostToDevice, L.s);
            coil_status sb = ea == cudaSuccess ? COIL_OK : COIL_ERR_CUDA;
            Launch Lg = L;
            Lg.d = bg->dd;
            if (sb == COIL_OK) sb = build_step_graph(c, 2, &Lg, bg, maxit);
            if (sb == COIL_OK && bg->exec) {
                c->batch = bg;
                fresh = true;
            } else {
                cudaGetLastError();
                if (bg->dd) cudaFree(bg->dd);
                if (bg->hstat) cudaFreeHost(bg->hstat);
                delete bg;
                c->graph_failed = true;                  // the same kernels, launched one by one
                c->err.clear();
            }
        }
        if (c->batch) {
            BatchGraph* bg = c->batch;
            cudaError_t e = fresh ? cudaSuccess
                                  : cudaMemcpyAsync(bg->dd, hd.data(), n * sizeof(CoilDev), cudaMemcpyHostToDevice, L.s);
            coil_status result = COIL_OK;
            for (long k = 0; k < n_steps && e == cudaSuccess && result == COIL_OK; ++k) {
                e = cudaGraphLaunch(bg->exec, L.s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(L.s);
                if (e != cudaSuccess) break;
                const int passes = bg->hstat[3 * n] > 0 ? bg->hstat[3 * n] : 1;
                c->launches += bg->fixed + (long long)bg->per_pass * passes;
                c->op_launches += 1 + passes;
                result = finish_step(bg->hstat);
            }
            if (e != cudaSuccess) return cuda_fail(c, e, "batch step");
            return result;
        }
    }
    // descriptors and the gathered status live in one device block per call
    CoilDev* dd = nullptr;
    int* dstat = nullptr;
    CK(cudaMalloc(&dd, n * sizeof(CoilDev) + 3 * n * sizeof(int)), "batch descriptors");
    dstat = reinterpret_cast<int*>(dd + n);
    std::vector<int> hstat(3 * (size_t)n);
    coil_status result = COIL_OK;
    cudaError_t e = cudaMemcpyAsync(dd, hd.data(), n * sizeof(CoilDev), cudaMemcpyHostToDevice, L.s);
    L.d = dd;
    for (long k = 0; k < n_steps && e == cudaSuccess && result == COIL_OK; ++k) {
        result = step_prologue(c, L);
        int chunk = 1;
        for (int i = 0; i < n; ++i) chunk = std::max(chunk, coils[i]->last_iters);
        int total = 0;
        bool all_done = false;
        while (result == COIL_OK) {
            for (int i = 0; i < chunk && result == COIL_OK; ++i) result = step_iteration(c, L);
            total += chunk;
            k_gather_status<<<(n + 127) / 128, 128, 0, L.s>>>(dd, n, dstat);
            e = cudaMemcpyAsync(hstat.data(), dstat, 3 * n * sizeof(int), cudaMemcpyDeviceToHost, L.s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(L.s);
            if (e != cudaSuccess) break;
            all_done = true;
            for (int i = 0; i < n; ++i) all_done = all_done && hstat[3 * i];
            if (all_done || total > maxit + 2) break;
            chunk = 1;
        }
        if (e != cudaSuccess || result != COIL_OK) break;
        harvest_events(c);
        result = step_epilogue(c, L);
        if (result == COIL_OK) result = finish_step(hstat.data());
    }
    cudaError_t e2 = cudaStreamSynchronize(L.s);
    cudaFree(dd);
    if (e != cudaSuccess) return cuda_fail(c, e, "batch step");
    if (e2 != cudaSuccess) return cuda_fail(c, e2, "batch step");
    return result;
}

coil_status coil_read_device(coil_t* c, const coil_drive* dr, double* dJ, double* dBr, double* dBz,
                             double* dT) {
    if (!c) return COIL_ERR_INVALID;
    cudaSetDevice(c->device);
    double Ba = host_drive_field(dr, c->t);
    const CoilDev& h = c->h;
    unsigned eb = (unsigned)((h.N + 255) / 256);
    cq::k_read<<<eb, 256, 0, c->stream>>>(c->d, Ba, dJ, dBr, dBz, dT);
    CK(cudaGetLastError(), "read");
    CK(cudaStreamSynchronize(c->stream), "read");
    return COIL_OK;
}

coil_status coil_read(coil_t* c, const coil_drive* dr, double* J, double* Br, double* Bz, double* T,
                      double* moment) {
    if (!c) return COIL_ERR_INVALID;
    cudaSetDevice(c->device);
    const CoilDev& h = c->h;
    double* buf = c->readbuf;
    size_t N = h.N;
    double Ba = host_drive_field(dr, c->t);
    unsigned eb = (unsigned)((N + 255) / 256);
    cq::k_read<<<eb, 256, 0, c->stream>>>(c->d, Ba, J ? buf : nullptr, Br ? buf + N : nullptr,
                                            Bz ? buf + 2 * N : nullptr, T ? buf + 3 * N : nullptr);
    const int mb = (int)std::min<size_t>(kMomentBlocks, (N + 255) / 256);
    cq::k_moment<<<mb, 256, 0, c->stream>>>(c->d, buf + 5 * N);
    cq::k_moment_sum<<<1, 32, 0, c->stream>>>(buf + 5 * N, mb, buf + 4 * N);
    cudaError_t e = cudaGetLastError();
    double* outs[4] = {J, Br, Bz, T};
    for (int k = 0; k < 4 && e == cudaSuccess; ++k)
        if (outs[k]) e = cudaMemcpyAsync(outs[k], buf + k * N, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    double mom = 0.0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&mom, buf + 4 * N, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "read");
    if (moment) *moment = mom;
    return COIL_OK;
}

coil_status coil_read_diag(coil_t* c, long first, long count, double* out) {
    if (!c) return COIL_ERR_INVALID;
    if (!out || first < 0 || count < 0 || first + count > c->steps)
        return fail(c, COIL_ERR_INVALID, "diagnostic range outside the completed steps");
    if (c->steps - first > c->h.diag_cap) return fail(c, COIL_ERR_INVALID, "records no longer in the ring");
    cudaSetDevice(c->device);
    for (long k = 0; k < count; ++k) {
        long slot = (first + k) % c->h.diag_cap;
        CK(cudaMemcpyAsync(out + k * COIL_DIAG_WIDTH, c->h.diag + slot * COIL_DIAG_WIDTH,
                           COIL_DIAG_WIDTH * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "diag");
    }
    CK(cudaStreamSynchronize(c->stream), "diag");
    return COIL_OK;
}

coil_status coil_read_onsets(coil_t* c, long* first_jump, long* first_quench) {
    if (!c) return COIL_ERR_INVALID;
    cudaSetDevice(c->device);
    size_t W = c->h.W;
    std::vector<long long> a(W), b(W);
    CK(cudaMemcpyAsync(a.data(), c->h.first_jump, W * 8, cudaMemcpyDeviceToHost, c->stream), "onsets");
    CK(cudaMemcpyAsync(b.data(), c->h.first_quench, W * 8, cudaMemcpyDeviceToHost, c->stream), "onsets");
    CK(cudaStreamSynchronize(c->stream), "onsets");
    for (size_t w = 0; w < W; ++w) {
        if (first_jump) first_jump[w] = (long)a[w];
        if (first_quench) first_quench[w] = (long)b[w];
    }
    return COIL_OK;
}

coil_status coil_read_wire_stats(coil_t* c, double* out) {
    if (!c || !out) return c ? fail(c, COIL_ERR_INVALID, "null buffer") : COIL_ERR_INVALID;
    cudaSetDevice(c->device);
    const size_t W = c->h.W;
    std::vector<long long> fr(W);
    CK(cudaMemcpyAsync(out, c->h.wstat, 6 * W * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "wire statistics");
    CK(cudaMemcpyAsync(fr.data(), c->h.first_rise, W * 8, cudaMemcpyDeviceToHost, c->stream), "wire statistics");
    CK(cudaStreamSynchronize(c->stream), "wire statistics");
    for (size_t w = 0; w < W; ++w) out[6 * W + w] = (double)fr[w];
    return COIL_OK;
}

coil_status coil_reset_wire_stats(coil_t* c) {
    if (!c) return COIL_ERR_INVALID;
    cudaSetDevice(c->device);
    return reset_wire_stats(c, true);
}

coil_status coil_get_currents(coil_t* c, double* I) {
    if (!c || !I) return c ? fail(c, COIL_ERR_INVALID, "null buffer") : COIL_ERR_INVALID;
    cudaSetDevice(c->device);
    CK(cudaMemcpyAsync(I, c->h.I, c->h.N * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "get");
    CK(cudaStreamSynchronize(c->stream), "get");
    return COIL_OK;
}

coil_status coil_set_currents(coil_t* c, const double* I) {
    if (!c || !I) return c ? fail(c, COIL_ERR_INVALID, "null buffer") : COIL_ERR_INVALID;
    for (int e = 0; e < c->h.N; ++e)
        if (!is_fin(I[e])) return fail(c, COIL_ERR_NONFINITE, "non-finite current");
    cudaSetDevice(c->device);
    const CoilDev& h = c->h;
    CK(cudaMemcpyAsync(h.I, I, h.N * sizeof(double), cudaMemcpyHostToDevice, c->stream), "set");
    TRY(apply_plain(c, h.I));
    CK(cudaMemcpyAsync(h.Phi, h.qv, h.N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "set");
    if (h.n_groups)    // injected currents carry no transport history: J_I restarts from 0
        CK(cudaMemsetAsync(h.Itr, 0, h.N * sizeof(double), c->stream), "set");
    CK(cudaMemsetAsync(h.x, 0, h.ld * sizeof(double), c->stream), "set");
    CK(cudaMemsetAsync(h.xprev, 0, h.N * sizeof(double), c->stream), "set");
    CK(cudaMemsetAsync(h.xprev2, 0, h.N * sizeof(double), c->stream), "set");
    CK(cudaStreamSynchronize(c->stream), "set");
    return COIL_OK;
}

coil_status coil_apply_operator(coil_t* c, const double* p, double* y) {
    if (!c || !p || !y) return c ? fail(c, COIL_ERR_INVALID, "null buffer") : COIL_ERR_INVALID;
    cudaSetDevice(c->device);
    const CoilDev& h = c->h;
    // keep the warm start: stash x in res
    CK(cudaMemcpyAsync(h.res, h.x, h.N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "apply");
    CK(cudaMemcpyAsync(h.zv, p, h.N * sizeof(double), cudaMemcpyHostToDevice, c->stream), "apply");
    TRY(apply_plain(c, h.zv));
    CK(cudaMemcpyAsync(y, h.qv, h.N * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "apply");
    CK(cudaMemcpyAsync(h.x, h.res, h.N * sizeof(double), cudaMemcpyDeviceToDevice, c->stream), "apply");
    CK(cudaStreamSynchronize(c->stream), "apply");
    return COIL_OK;
}

coil_status coil_read_operator(coil_t* c, double* M) {
    if (!c || !M) return c ? fail(c, COIL_ERR_INVALID, "null buffer") : COIL_ERR_INVALID;
    cudaSetDevice(c->device);
    const CoilDev& h = c->h;
    size_t N = h.N, ld = h.ld;
    size_t esz = h.precision == PREC_FP64 ? 8 : (h.precision == PREC_FP32 ? 4 : 2);
    std::vector<unsigned char> row(ld * esz);
    if (h.op_format == 1) {
        size_t C = h.C, NT = h.NT;
        std::vector<float> tab(C * C * (2 * NT - 1));
        CK(cudaMemcpy(tab.data(), h.tab32, tab.size() * sizeof(float), cudaMemcpyDeviceToHost), "read operator");
        for (size_t i = 0; i < N; ++i)
            for (size_t j = 0; j < N; ++j) {
                long long d = (long long)(i / C) - (long long)(j / C);
                M[i * N + j] = tab[(size_t)(d + (long long)NT - 1) * C * C + (i % C) * C + (j % C)];
            }
    }
    if (h.op_format == 2) {
        // (hi + lo) 2^-exT of the split FP16 table [half][offset >= 0][k block][c][64];
        // offset d < 0 reads T_{-d} transposed
        const TcShape& sh = c->tc->sh;
        size_t C = sh.C, nkb = sh.n_kb;
        size_t half_n = tc_table_halves(sh) / 2;
        std::vector<__half> t16(2 * half_n);
        CK(cudaMemcpy(t16.data(), c->tc->t16, t16.size() * sizeof(__half), cudaMemcpyDeviceToHost),
           "read operator");
        const double inv = ldexp(1.0, -c->tc->exT);
        for (size_t i = 0; i < N; ++i)
            for (size_t j = 0; j < N; ++j) {
                long long d = (long long)(i / C) - (long long)(j / C);
                size_t ci = d >= 0 ? i % C : j % C, cj = d >= 0 ? j % C : i % C;
                size_t k = (((size_t)(d >= 0 ? d : -d) * nkb + cj / 64) * C + ci) * 64 + cj % 64;
                M[i * N + j] = ((double)__half2float(t16[k]) + (double)__half2float(t16[half_n + k])) * inv;
            }
    }
    for (size_t i = 0; i < N && h.op_format == 0; ++i) {
        CK(cudaMemcpy(row.data(), (const unsigned char*)h.Mfar + i * ld * esz, ld * esz, cudaMemcpyDeviceToHost),
           "read operator");
        for (size_t j = 0; j < N; ++j) {
            double v;
            if (esz == 8) {
                memcpy(&v, &row[j * 8], 8);
            } else if (esz == 4) {
                float f;
                memcpy(&f, &row[j * 4], 4);
                v = f;
            } else {
                unsigned short b;
                memcpy(&b, &row[j * 2], 2);
                unsigned u = (unsigned)b << 16;
                float f;
                memcpy(&f, &u, 4);
                v = f;
            }
            M[i * N + j] = v;
        }
    }
    std::vector<double> nb((size_t)h.n_types * h.B * h.B);
    std::vector<int> bt(h.W);
    CK(cudaMemcpy(nb.data(), h.near, nb.size() * 8, cudaMemcpyDeviceToHost), "read operator");
    CK(cudaMemcpy(bt.data(), h.block_type, bt.size() * 4, cudaMemcpyDeviceToHost), "read operator");
    for (int w = 0; w < h.W; ++w)
        for (int a = 0; a < h.B; ++a)
            for (int b = 0; b < h.B; ++b)
                M[(size_t)(w * h.B + a) * N + w * h.B + b] += nb[((size_t)bt[w] * h.B + a) * h.B + b];
    return COIL_OK;
}

// "COILST04": state of I, Phi, x, xprev, xprev2, u_T, onsets and per-wire statistics
constexpr unsigned long long kStateMagic = 0x434f494c53543034ULL;

struct StateHeader {
    unsigned long long magic;
    long long N, W, G, steps;
    double t;
};

coil_status coil_save_state(coil_t* c, void* buf, size_t* bytes) {
    if (!c || !bytes) return c ? fail(c, COIL_ERR_INVALID, "null size pointer") : COIL_ERR_INVALID;
    const CoilDev& h = c->h;
    size_t N = h.N, W = h.W, G = (size_t)h.Gr * h.Gz;
    const size_t NI = h.n_groups ? N : 0;   // transport part J_I with subelements
    size_t need = sizeof(StateHeader) + (5 * N + G + 6 * W + NI) * sizeof(double) + 3 * W * sizeof(long long);
    if (!buf) { *bytes = need; return COIL_OK; }
    if (*bytes < need) return fail(c, COIL_ERR_INVALID, "state buffer too small");
    cudaSetDevice(c->device);
    StateHeader hd{kStateMagic, (long long)N, (long long)W, (long long)G, c->steps, c->t};
    unsigned char* p = (unsigned char*)buf;
    memcpy(p, &hd, sizeof(hd));
    p += sizeof(hd);
    CK(cudaMemcpy(p, h.I, N * 8, cudaMemcpyDeviceToHost), "save"); p += N * 8;
    CK(cudaMemcpy(p, h.Phi, N * 8, cudaMemcpyDeviceToHost), "save"); p += N * 8;
    CK(cudaMemcpy(p, h.x, N * 8, cudaMemcpyDeviceToHost), "save"); p += N * 8;
    CK(cudaMemcpy(p, h.xprev, N * 8, cudaMemcpyDeviceToHost), "save"); p += N * 8;
    CK(cudaMemcpy(p, h.xprev2, N * 8, cudaMemcpyDeviceToHost), "save"); p += N * 8;
    if (G) { CK(cudaMemcpy(p, h.uT, G * 8, cudaMemcpyDeviceToHost), "save"); p += G * 8; }
    CK(cudaMemcpy(p, h.first_jump, W * 8, cudaMemcpyDeviceToHost), "save"); p += W * 8;
    CK(cudaMemcpy(p, h.first_quench, W * 8, cudaMemcpyDeviceToHost), "save"); p += W * 8;
    CK(cudaMemcpy(p, h.first_rise, W * 8, cudaMemcpyDeviceToHost), "save"); p += W * 8;
    CK(cudaMemcpy(p, h.wstat, 6 * W * 8, cudaMemcpyDeviceToHost), "save"); p += 6 * W * 8;
    if (NI) CK(cudaMemcpy(p, h.Itr, NI * 8, cudaMemcpyDeviceToHost), "save");
    *bytes = need;
    return COIL_OK;
}

coil_status coil_load_state(coil_t* c, const void* buf, size_t bytes) {
    if (!c || !buf) return c ? fail(c, COIL_ERR_INVALID, "null state buffer") : COIL_ERR_INVALID;
    const CoilDev& h = c->h;
    size_t N = h.N, W = h.W, G = (size_t)h.Gr * h.Gz;
    const size_t NI = h.n_groups ? N : 0;   // transport part J_I with subelements
    size_t need = sizeof(StateHeader) + (5 * N + G + 6 * W + NI) * sizeof(double) + 3 * W * sizeof(long long);
    StateHeader hd;
    if (bytes < need) return fail(c, COIL_ERR_INVALID, "state buffer too small");
    memcpy(&hd, buf, sizeof(hd));
    if (hd.magic != kStateMagic || hd.N != (long long)N || hd.W != (long long)W || hd.G != (long long)G)
        return fail(c, COIL_ERR_INVALID, "state does not belong to a coil of this shape");
    cudaSetDevice(c->device);
    const unsigned char* p = (const unsigned char*)buf + sizeof(hd);
    CK(cudaMemcpy(h.I, p, N * 8, cudaMemcpyHostToDevice), "load"); p += N * 8;
    CK(cudaMemcpy(h.Phi, p, N * 8, cudaMemcpyHostToDevice), "load"); p += N * 8;
    CK(cudaMemcpy(h.x, p, N * 8, cudaMemcpyHostToDevice), "load"); p += N * 8;
    CK(cudaMemcpy(h.xprev, p, N * 8, cudaMemcpyHostToDevice), "load"); p += N * 8;
    CK(cudaMemcpy(h.xprev2, p, N * 8, cudaMemcpyHostToDevice), "load"); p += N * 8;
    if (G) { CK(cudaMemcpy(h.uT, p, G * 8, cudaMemcpyHostToDevice), "load"); p += G * 8; }
    CK(cudaMemcpy(h.first_jump, p, W * 8, cudaMemcpyHostToDevice), "load"); p += W * 8;
    CK(cudaMemcpy(h.first_quench, p, W * 8, cudaMemcpyHostToDevice), "load"); p += W * 8;
    CK(cudaMemcpy(h.first_rise, p, W * 8, cudaMemcpyHostToDevice), "load"); p += W * 8;
    CK(cudaMemcpy(h.wstat, p, 6 * W * 8, cudaMemcpyHostToDevice), "load"); p += 6 * W * 8;
    if (NI) CK(cudaMemcpy(h.Itr, p, NI * 8, cudaMemcpyHostToDevice), "load");
    Scalars sc;
    CK(cudaMemcpy(&sc, h.sc, sizeof(sc), cudaMemcpyDeviceToHost), "load");
    sc.t = hd.t;
    sc.step = hd.steps;
    CK(cudaMemcpy(h.sc, &sc, sizeof(sc), cudaMemcpyHostToDevice), "load");
    c->t = hd.t;
    c->steps = hd.steps;
    return COIL_OK;
}

coil_status coil_info(const coil_t* c, coil_info_t* info) {
    if (!c || !info) return COIL_ERR_INVALID;
    info->n_elem = c->h.N;
    info->n_blocks = c->h.W;
    info->block = c->h.B;
    info->grid_r = c->h.Gr;
    info->grid_z = c->h.Gz;
    info->precision = c->h.precision;
    info->operator_bytes = c->op_bytes;
    info->device_bytes = c->bytes;
    info->steps = c->steps;
    info->t = c->t;
    info->setup_ms = c->setup_ms;
    info->kernel_launches = c->launches;
    info->operator_launches = c->op_launches;
    info->operator_ms = c->op_ms;
    info->pcg_iterations = c->pcg_iters;
    info->descriptor_bytes = sizeof(CoilDev);
    info->step_graph = c->step_exec ? 1 : 0;
    return COIL_OK;
}

coil_status coil_tc_schedule(const coil_t* c, int* mode, int* n_cta, int* stages, double* us) {
    if (!c) return COIL_ERR_INVALID;
    if (!c->tc) return fail(const_cast<coil_t*>(c), COIL_ERR_INVALID, "not the tensor-core Toeplitz format");
    if (mode) *mode = c->tc->sh.mode;
    if (n_cta) *n_cta = c->tc->sh.n_cta;
    if (stages) *stages = c->tc->sh.stages;
    if (us) *us = c->tc->tuned_us;
    return COIL_OK;
}

coil_status coil_tc_candidates(const coil_t* c, int* count, double* out) {
    if (!c || !count) return COIL_ERR_INVALID;
    if (!c->tc) return fail(const_cast<coil_t*>(c), COIL_ERR_INVALID, "not the tensor-core Toeplitz format");
    const int n = (int)c->tc->tuned.size();
    if (out) {
        const int m = std::min(n, *count);
        for (int i = 0; i < m; ++i) {
            const TcPlan::Tuned& t = c->tc->tuned[i];
            out[4 * i] = t.mode;
            out[4 * i + 1] = t.n_cta;
            out[4 * i + 2] = t.stages;
            out[4 * i + 3] = t.us;
        }
    }
    *count = n;
    return COIL_OK;
}

coil_status coil_set_tc_schedule(coil_t* c, int mode, int n_cta, int stages) {
    if (!c) return COIL_ERR_INVALID;
    if (!c->tc) return fail(c, COIL_ERR_INVALID, "not the tensor-core Toeplitz format");
    cudaSetDevice(c->device);
    if (mode == -1) return tc_autotune(c, true);
    const TcShape& cur = c->tc->sh;
    TcShape sh;
    bool ok = false;
    if (mode == 0) {
        ok = tc_shape(cur.C, cur.NT, c->n_sm, &sh);
        if (ok && stages > 0) {
            if (stages > sh.stages || stages < sh.n_acc) ok = false;
            else sh.stages = stages;
        }
        if (ok && n_cta > 0) ok = false;          // the two-fill apply sizes its own grid
    } else if (mode == 1) {
        ok = tc2_shape(cur.C, cur.NT, c->n_sm, n_cta > 0 ? n_cta : 0, stages > 0 ? stages : 0, &sh) &&
             (stages <= 0 || sh.stages == stages);
    }
    if (!ok) return fail(c, COIL_ERR_INVALID, "unsupported tensor-core schedule for this coil");
    TRY(tc_plan_schedule(c, sh));
    double us = 0.0;
    TRY(tc_time_apply(c, &us));
    c->tc->tuned_us = us;
    c->tc->tuned_sh = c->tc->sh;      // kept when the coil steps alone after batched steps
    c->tc->in_batch = false;
    return COIL_OK;
}

coil_status coil_set_wait_limit(coil_t* c, long long cycles) {
    if (!c) return COIL_ERR_INVALID;
    if (cycles < 0) return fail(c, COIL_ERR_INVALID, "wait limit must be >= 0");
    cudaSetDevice(c->device);
    const long long v = cycles;
    CK(cudaMemcpyAsync(&c->h.sc->tc_wait, &v, sizeof(v), cudaMemcpyHostToDevice, c->stream), "wait limit");
    CK(cudaStreamSynchronize(c->stream), "wait limit");
    return COIL_OK;
}

coil_status coil_reset_counters(coil_t* c) {
    if (!c) return COIL_ERR_INVALID;
    c->launches = c->op_launches = c->pcg_iters = 0;
    c->op_ms = 0.0;
    return COIL_OK;
}

const char* coil_last_error(const coil_t* c) {
    if (!c) return kNoHandle;
    return c->err.c_str();
}

void coil_destroy(coil_t* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (void* p : c->allocs) cudaFree(p);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (cudaStream_t st : c->aux) cudaStreamDestroy(st);
    if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
    if (c->adj_exec) cudaGraphExecDestroy(c->adj_exec);
    if (c->replay_exec) cudaGraphExecDestroy(c->replay_exec);
    if (c->batch) {
        if (c->batch->exec) cudaGraphExecDestroy(c->batch->exec);
        cudaFree(c->batch->dd);
        cudaFreeHost(c->batch->hstat);
        delete c->batch;
    }
    if (c->tcb) {
        tc_batch_free(c->tcb);
        delete c->tcb;
    }
    if (c->body_stream) cudaStreamDestroy(c->body_stream);
    for (cudaEvent_t e : c->aux_ev) cudaEventDestroy(e);
    if (c->d) cudaFree(c->d);
    delete c->tc;
    if (c->pinned) cudaFreeHost(c->pinned);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"

// ---- internal view for entry points in other translation units
#include "internal.h"

namespace cq {
bool coil_view(const coil_t* c, CoilView* v) {
    if (!c || !v) return false;
    v->host = &c->h;
    v->dev = c->d;
    v->device = c->device;
    v->n_sm = c->n_sm;
    return true;
}

coil_status coil_set_error(coil_t* c, coil_status st, const char* msg) {
    if (c) c->err = msg;
    return st;
}
}  // namespace cq

// ---- adjoint driver -----------------------------------------------------
namespace cq {
struct AdjBufs {
    double* lamI;
    const double* lamI_next;
    double* lamU;
    const double* lamU_next;
    double* a;
    double* b;
    double* lamQ;
    double* lamBr;
    double* lamBz;
    const double* xk;
    double* g_f;
    double* gparts;
};
void launch_adj_thermal(const CoilDev* d, const CoilDev& h, const AdjBufs& ab, cudaStream_t s);
void launch_adj_setup(const CoilDev* d, const CoilDev& h, const AdjBufs& ab, cudaStream_t s);
void launch_adj_mult_pointwise(const CoilDev* d, const CoilDev& h, const AdjBufs& ab, double wP, cudaStream_t s);
void launch_adj_stencil_t(const CoilDev* d, const CoilDev& h, const AdjBufs& ab, cudaStream_t s);
void launch_adj_near(const CoilDev* d, const CoilDev& h, cudaStream_t s);
void launch_adj_accum(const CoilDev* d, const CoilDev& h, const AdjBufs& ab, double wk, int with_field,
                      cudaStream_t s);
void launch_adj_seed(const CoilDev* d, const CoilDev& h, double* lamI, double wk, cudaStream_t s);
void launch_adj_reduce(const CoilDev* d, const double* gparts, double* out, cudaStream_t s);
}  // namespace cq

namespace {

// Device scratch of one adjoint call, released when the call returns.
struct AdjMem {
    std::vector<void*> ptrs;
    coil_t* c;
    explicit AdjMem(coil_t* cc) : c(cc) {}
    ~AdjMem() {
        for (void* p : ptrs) cudaFree(p);
    }
    coil_status get(double** p, size_t n, const char* what) {
        void* v = nullptr;
        cudaError_t e = cudaMalloc(&v, (n ? n : 1) * sizeof(double));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, COIL_ERR_OOM, std::string("adjoint: allocation of ") + what + " failed");
        }
        ptrs.push_back(v);
        *p = static_cast<double*>(v);
        CK(cudaMemsetAsync(v, 0, (n ? n : 1) * sizeof(double), c->stream), "adjoint memset");
        return COIL_OK;
    }
};

// Copy the stepping state (I, flux, warm start, T^4) to or from `slot`.
coil_status state_copy(coil_t* c, double* slot, bool save, bool with_x) {
    const CoilDev& h = c->h;
    size_t N = h.N, G = (size_t)h.Gr * h.Gz;
    cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
    double* parts[6] = {h.I, h.Phi, h.x, h.xprev, h.xprev2, h.uT};
    size_t sizes[6] = {N, N, N, N, N, G};
    size_t off = 0;
    for (int i = 0; i < 6; ++i) {
        if (sizes[i] && ((i < 2 || i > 4) || with_x)) {
            if (save) CK(cudaMemcpyAsync(slot + off, parts[i], sizes[i] * 8, k, c->stream), "state copy");
            else CK(cudaMemcpyAsync(parts[i], slot + off, sizes[i] * 8, k, c->stream), "state copy");
        }
        off += sizes[i];
    }
    return COIL_OK;
}

coil_status set_device_time(coil_t* c, double t, long long step) {
    // a pageable source: the copy is staged before cudaMemcpyAsync returns
    struct { double t; long long step; } ts = {t, step};
    CK(cudaMemcpyAsync(c->h.sc, &ts, sizeof(ts), cudaMemcpyHostToDevice, c->stream), "time");
    return COIL_OK;
}

// The transposed KKT solve of one reverse step: the same projected PCG with
// the right-hand side prepared by k_adj_setup (k_pointwise already ran).
coil_status adjoint_prologue(coil_t* c, const Launch& L) {
    c->launches += launch_factor(L, true);
    c->launches += scale_reduce(L);
    TRY(gemv(c, L, 0));
    c->launches += launch_near(L, 0, true);
    c->launches += launch_init(L, true, true);
    c->launches += init_reduce(L);
    CK(cudaGetLastError(), "adjoint solve");
    return COIL_OK;
}

coil_status adjoint_status(coil_t* c) {
    int st = c->pinned->status;
    if (st == ST_KERNEL) return fail(c, COIL_ERR_CUDA, tc_timeout_text(c));
    if (!c->pinned->done || st == ST_NOT_CONVERGED)
        return fail(c, COIL_ERR_NOT_CONVERGED, "adjoint solve did not converge within maxit iterations");
    if (st == ST_NONFINITE) return fail(c, COIL_ERR_NONFINITE, "non-finite value in the adjoint solve");
    c->pcg_iters += c->pinned->iter;
    return COIL_OK;
}

coil_status adjoint_solve(coil_t* c) {
    const CoilDev& h = c->h;
    if (!c->profile && !c->graph_failed) {
        // one graph: the prologue, then the PCG loop the device ends
        if (!c->adj_exec && build_step_graph(c, 1) != COIL_OK) {
            c->graph_failed = true;                      // the same kernels, launched one by one
            c->err.clear();
        }
        if (c->adj_exec) {
            CK(cudaGraphLaunch(c->adj_exec, c->stream), "adjoint graph launch");
            CK(cudaStreamSynchronize(c->stream), "adjoint solve");
            const int passes = c->pinned->passes > 0 ? c->pinned->passes : 1;
            c->launches += c->adj_fixed + (long long)c->adj_per_pass * passes;
            c->op_launches += 1 + passes;
            return adjoint_status(c);
        }
    }
    Launch L = single_launch(c);
    TRY(adjoint_prologue(c, L));
    int chunk = !c->profile && c->last_iters > 1 ? c->last_iters : 1;
    int total = 0;
    for (;;) {
        for (int i = 0; i < chunk; ++i) TRY(step_iteration(c, L));
        total += chunk;
        TRY(read_scalars(c));
        if (c->pinned->done) break;
        if (total > h.maxit + 2) break;
        chunk = 1;
    }
    harvest_events(c);
    return adjoint_status(c);
}

}  // namespace

extern "C" coil_status coil_set_params(coil_t* c, const double* jc_factor, double n, double C_eps) {
    if (!c) return COIL_ERR_INVALID;
    if (!is_fin(n) || !(n >= 1.0) || !is_fin(C_eps)) return fail(c, COIL_ERR_INVALID, "n must be >= 1, C_eps finite");
    cudaSetDevice(c->device);
    if (jc_factor) {
        for (int e = 0; e < c->h.N; ++e)
            if (!is_fin(jc_factor[e]) || jc_factor[e] < 0.0)
                return fail(c, COIL_ERR_NONFINITE, "non-finite or negative jc_factor");
        CK(cudaMemcpyAsync((void*)c->h.jc_factor, jc_factor, c->h.N * sizeof(double), cudaMemcpyHostToDevice,
                           c->stream), "set params");
    }
    c->h.nexp = n;
    c->h.C_eps = C_eps;
    round_constants(c->h);
    TRY(sync_descriptor(c));
    CK(cudaStreamSynchronize(c->stream), "set params");
    return COIL_OK;
}

extern "C" coil_status coil_adjoint(coil_t* c, long n_steps, const coil_drive* drive, int ckpt_every,
                                    const double* dL_dm, double* g_jc_factor, double* g_n, double* g_C_eps) {
    if (c && !dL_dm) return fail(c, COIL_ERR_INVALID, "adjoint needs dL_dm");
    return coil_adjoint_losses(c, n_steps, drive, ckpt_every, dL_dm, nullptr, g_jc_factor, g_n, g_C_eps);
}

extern "C" coil_status coil_adjoint_losses(coil_t* c, long n_steps, const coil_drive* drive, int ckpt_every,
                                           const double* dL_dm, const double* dL_dP, double* g_jc_factor,
                                           double* g_n, double* g_C_eps) {
    if (!c) return COIL_ERR_INVALID;
    if (n_steps < 1 || ckpt_every < 1 || (!dL_dm && !dL_dP))
        return fail(c, COIL_ERR_INVALID, "adjoint needs n_steps >= 1, ckpt_every >= 1 and dL_dm or dL_dP");
    if (c->h.n_groups) return fail(c, COIL_ERR_INVALID, "the adjoint does not differentiate the subelement decoupling");
    for (long k = 0; k < n_steps; ++k)
        if ((dL_dm && !is_fin(dL_dm[k])) || (dL_dP && !is_fin(dL_dP[k])))
            return fail(c, COIL_ERR_NONFINITE, "non-finite dL/dm or dL/dP");
    auto wm = [&](long k) { return dL_dm ? dL_dm[k] : 0.0; };
    cudaSetDevice(c->device);
    TRY(set_drive(c, drive));
    CoilDev& h = c->h;
    const size_t N = h.N, G = (size_t)h.Gr * h.Gz, W = h.W;
    const size_t S = 5 * N + G;                       // one stored state: I, Phi, x, xprev, xprev2, u_T
    const long nseg = (n_steps + ckpt_every - 1) / ckpt_every;
    const bool grid = h.has_grid != 0, thermal = h.thermal != 0;
    cudaStream_t s = c->stream;
    AdjMem mem(c);
    double *ck, *seg, *fin, *lamA, *lamB, *lamUA, *lamUB, *abuf, *bbuf, *lamQ, *lamBr, *lamBz, *gf, *gparts, *musave,
        *out2;
    TRY(mem.get(&ck, nseg * S, "checkpoints"));
    TRY(mem.get(&seg, (size_t)ckpt_every * S, "segment states"));
    TRY(mem.get(&fin, S, "final state"));
    TRY(mem.get(&lamA, N, "lambda_I"));
    TRY(mem.get(&lamB, N, "lambda_I"));
    TRY(mem.get(&lamUA, G, "lambda_u"));
    TRY(mem.get(&lamUB, G, "lambda_u"));
    TRY(mem.get(&abuf, G, "reverse ADI"));
    TRY(mem.get(&bbuf, G, "reverse ADI"));
    TRY(mem.get(&lamQ, G, "lambda_q"));
    TRY(mem.get(&lamBr, N, "lambda_B"));
    TRY(mem.get(&lamBz, N, "lambda_B"));
    TRY(mem.get(&gf, N, "dL/df"));
    TRY(mem.get(&gparts, 2 * W, "partials"));
    TRY(mem.get(&musave, N, "mu"));
    TRY(mem.get(&out2, 2, "outputs"));
    double *muprev, *muprev2;
    TRY(mem.get(&muprev, N, "previous adjoint solution"));
    TRY(mem.get(&muprev2, N, "previous adjoint solution"));
    // records of every forward step's solve outputs (x, residual, loop
    // voltages), so that the recomputation of a segment replays its steps
    // without solving them; left out (the recomputation then solves) when they
    // would take more than a quarter of the free device memory or 4 GiB
    bool replay = false;
    double *rx = nullptr, *rres = nullptr, *ruw = nullptr, *ru = nullptr;
    if (nseg > 1) {
        size_t free_b = 0, total_b = 0;
        const size_t want = (size_t)n_steps * (2 * N + 2 * W) * sizeof(double);
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && want <= free_b / 4 && want <= (size_t(4) << 30)) {
            replay = mem.get(&rx, (size_t)n_steps * N, "step records") == COIL_OK &&
                     mem.get(&rres, (size_t)n_steps * N, "step records") == COIL_OK &&
                     mem.get(&ruw, (size_t)n_steps * W, "step records") == COIL_OK &&
                     mem.get(&ru, (size_t)n_steps * W, "step records") == COIL_OK;
            if (!replay) c->err.clear();
        }
    }

    // forward pass, checkpoint every ckpt_every steps; the states of the last
    // segment are kept as they are made, so that segment needs no recomputation
    std::vector<double> t_ck(nseg);
    std::vector<long long> st_ck(nseg);
    const long k0_last = (nseg - 1) * ckpt_every;
    std::vector<double> t_last(n_steps - k0_last);
    const size_t xoff = 2 * N;                      // position of the warm start / Idot in a slot
    if (replay) {
        // the device's step index is the record index's origin
        TRY(set_device_time(c, c->t, c->steps));
        h.rec_x = rx;
        h.rec_res = rres;
        h.rec_uw = ruw;
        h.rec_u = ru;
        h.rec_step0 = c->steps;
        h.rec_mode = 1;
        TRY(sync_descriptor(c));
    }
    for (long k = 0; k < n_steps; ++k) {
        if (k % ckpt_every == 0) {
            TRY(state_copy(c, ck + (k / ckpt_every) * S, true, true));
            t_ck[k / ckpt_every] = c->t;
            st_ck[k / ckpt_every] = c->steps;
        }
        double* slot = k >= k0_last ? seg + (k - k0_last) * S : nullptr;
        if (slot) {
            TRY(state_copy(c, slot, true, false));
            t_last[k - k0_last] = c->t;
        }
        TRY(run_step(c));
        if (slot) CK(cudaMemcpyAsync(slot + xoff, h.x, N * 8, cudaMemcpyDeviceToDevice, s), "adjoint");
    }
    if (replay) {
        h.rec_mode = 0;
        TRY(sync_descriptor(c));
    }
    TRY(state_copy(c, fin, true, true));
    const double t_fin = c->t;
    const long long st_fin = c->steps;
    const int last_iters_fin = c->last_iters;

    // reverse sweep: its pointwise launches recompute steps already counted,
    // so the per-wire statistics stay as the forward pass left them.  Its
    // transposed solves extrapolate quadratically from their own last three
    // solutions (history in muprev, muprev2); the recomputed forward steps use
    // the forward history, as the forward pass did.
    double* const xprev_fwd = h.xprev;
    double* const xprev2_fwd = h.xprev2;
    struct AccGuard {
        coil_t* c;
        double *xp, *xp2;
        ~AccGuard() {
            c->h.acc_on = 1;
            c->h.extrap = 1;
            c->h.xprev = xp;
            c->h.xprev2 = xp2;
            c->h.rec_mode = 0;
            c->h.rec_x = c->h.rec_res = c->h.rec_uw = c->h.rec_u = nullptr;
            sync_descriptor(c);
        }
    } acc_guard{c, xprev_fwd, xprev2_fwd};
    h.acc_on = 0;
    TRY(sync_descriptor(c));
    long solved = 0;                                 // transposed solves done
    double* lamI_next = lamA;
    double* lamI = lamB;
    double* lamU_next = lamUA;
    double* lamU = lamUB;
    launch_adj_seed(c->d, h, lamI_next, wm(n_steps - 1), s);
    CK(cudaMemsetAsync(h.x, 0, h.ld * sizeof(double), s), "adjoint");
    for (long sg = nseg - 1; sg >= 0; --sg) {
        long k0 = sg * ckpt_every, k1 = std::min<long>(n_steps, k0 + ckpt_every);
        std::vector<double> t_k(k1 - k0);
        if (sg == nseg - 1) {
            t_k = t_last;                           // kept from the forward pass
        } else {
            CK(cudaMemcpyAsync(musave, h.x, N * 8, cudaMemcpyDeviceToDevice, s), "adjoint");
            h.extrap = 1;
            h.xprev = xprev_fwd;
            h.xprev2 = xprev2_fwd;
            h.rec_mode = replay ? 2 : 0;
            TRY(sync_descriptor(c));
            TRY(state_copy(c, ck + sg * S, false, true));
            c->t = t_ck[sg];
            c->steps = st_ck[sg];
            TRY(set_device_time(c, c->t, c->steps));
            for (long k = k0; k < k1; ++k) {
                double* slot = seg + (k - k0) * S;
                TRY(state_copy(c, slot, true, false));
                t_k[k - k0] = c->t;
                TRY(replay ? run_replay_step(c) : run_step(c));
                CK(cudaMemcpyAsync(slot + xoff, h.x, N * 8, cudaMemcpyDeviceToDevice, s), "adjoint");
            }
            if (replay) {
                h.rec_mode = 0;
                TRY(sync_descriptor(c));
            }
            CK(cudaMemcpyAsync(h.x, musave, N * 8, cudaMemcpyDeviceToDevice, s), "adjoint");
        }
        h.xprev = muprev;
        h.xprev2 = muprev2;
        for (long k = k1 - 1; k >= k0; --k) {
            double* slot = seg + (k - k0) * S;
            TRY(state_copy(c, slot, false, false));
            TRY(set_device_time(c, t_k[k - k0], st_ck[sg] + (k - k0)));
            AdjBufs ab{lamI, lamI_next, lamU, lamU_next, abuf, bbuf, lamQ, lamBr, lamBz, slot + xoff, gf, gparts};
            c->launches += launch_pointwise(single_launch(c));
            if (thermal) launch_adj_thermal(c->d, h, ab, s);
            launch_adj_setup(c->d, h, ab, s);
            CK(cudaGetLastError(), "adjoint launch");
            const int mode = solved >= 3 ? 4 : (solved == 2 ? 6 : 5);
            if (h.extrap != mode) {
                h.extrap = mode;
                TRY(sync_descriptor(c));
            }
            TRY(adjoint_solve(c));
            ++solved;
            launch_adj_mult_pointwise(c->d, h, ab, dL_dP ? dL_dP[k] : 0.0, s);
            if (grid) {
                launch_adj_stencil_t(c->d, h, ab, s);
                Launch L = single_launch(c);
                L.need_q = true;                     // k_adj_near reads q
                TRY(gemv(c, L, 1));
                launch_adj_near(c->d, h, s);
            }
            launch_adj_accum(c->d, h, ab, k >= 1 ? wm(k - 1) : 0.0, grid ? 1 : 0, s);
            c->launches += 5;
            CK(cudaGetLastError(), "adjoint launch");
            std::swap(lamI, lamI_next);
            std::swap(lamU, lamU_next);
        }
    }
    launch_adj_reduce(c->d, gparts, out2, s);
    double g2[2] = {0.0, 0.0};
    CK(cudaMemcpyAsync(g2, out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s), "adjoint");
    if (g_jc_factor) CK(cudaMemcpyAsync(g_jc_factor, gf, N * 8, cudaMemcpyDeviceToHost, s), "adjoint");
    CK(cudaStreamSynchronize(s), "adjoint");
    if (g_n) *g_n = g2[0];
    if (g_C_eps) *g_C_eps = g2[1];
    // back to the state after the forward steps
    h.extrap = 1;
    h.xprev = xprev_fwd;
    h.xprev2 = xprev2_fwd;
    TRY(sync_descriptor(c));
    TRY(state_copy(c, fin, false, true));
    c->t = t_fin;
    c->steps = st_fin;
    c->last_iters = last_iters_fin;
    TRY(set_device_time(c, t_fin, st_fin));
    return COIL_OK;
}
