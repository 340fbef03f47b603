// api.cu -- the C ABI (comet.h): problem lifetime, host/device buffer
// staging and the launch of the persistent evaluator.

#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "comet.h"
#include "comet_internal.h"
#include "problem_internal.h"

namespace {

thread_local std::string g_err;

comet_status fail(comet_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

comet_status cuda_fail(cudaError_t e, const char* what) {
    return fail(e == cudaErrorMemoryAllocation ? COMET_ERR_OOM : COMET_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define CUDA_TRY(call, what)                        \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// true if ptr is device (or managed) memory usable in place by kernels
bool is_device_ptr(const void* ptr) {
    if (!ptr) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Internal scaling of the dynamics rows: the median over the four faces of
// the Jacobian-row norm of d_k,r with respect to (x_k, u_k, x_{k+1}) at the
// cold-start reference point (zero controls, s = 0, theta = 0); the paper
// scales rows by their median Jacobian-row norm over sample orders.
void dynamics_row_scales(const comet_instance_desc& d, double sigma[4]) {
    const double dt = d.dt, k = d.kappa, ic2 = 1.0 / (d.c_ls * d.c_ls);
    for (int r = 0; r < 4; ++r) {
        double nrm[4];
        for (int face = 0; face < 4; ++face) {
            const double nx = (face == 0) ? 1.0 : ((face == 2) ? -1.0 : 0.0);
            const double ny = (face == 1) ? 1.0 : ((face == 3) ? -1.0 : 0.0);
            const double tx = -ny, ty = nx;
            const double a = (face % 2 == 0) ? 0.5 * d.side_x : 0.5 * d.side_y;
            // d f_r / d u at the reference point (theta = 0, s = 0, u = 0);
            // d f / d x vanishes there
            double fu[3] = {0, 0, 0};
            if (r == 0) { fu[0] = k * nx; fu[1] = k * tx; }
            if (r == 1) { fu[0] = k * ny; fu[1] = k * ty; }
            if (r == 2) { fu[1] = -k * a * ic2; }
            if (r == 3) { fu[2] = 1.0; }
            double s2 = 2.0;  // -1 on x_k,r and +1 on x_{k+1},r
            for (int j = 0; j < 3; ++j) s2 += dt * dt * fu[j] * fu[j];
            nrm[face] = sqrt(s2);
        }
        std::sort(nrm, nrm + 4);
        sigma[r] = 0.5 * (nrm[1] + nrm[2]);
    }
}

}  // namespace

namespace comet {

// FP32 / FP64 device constants of one instance descriptor.
void make_dev_instance(const comet_instance_desc& d, DevInstance* out) {
    DevInstance& q = *out;
    memset(&q, 0, sizeof(q));
    double sigma[4];
    dynamics_row_scales(d, sigma);
    q.dt_d = d.dt;
    q.kappa_d = d.kappa;
    q.inv_c2_d = 1.0 / (d.c_ls * d.c_ls);
    q.mu_d = d.mu;
    q.sc_cone_d = 1.0 / sqrt(1.0 + d.mu * d.mu);
    for (int f = 0; f < 4; ++f) {
        q.a_d[f] = (f % 2 == 0) ? 0.5 * d.side_x : 0.5 * d.side_y;
        q.ell_d[f] = (f % 2 == 0) ? 0.5 * d.side_y : 0.5 * d.side_x;
        q.a[f] = (float)q.a_d[f];
        q.ell[f] = (float)q.ell_d[f];
    }
    for (int r = 0; r < 4; ++r) {
        q.sigma_d[r] = sigma[r];
        q.inv_sigma[r] = (float)(1.0 / sigma[r]);
    }
    for (int j = 0; j < 3; ++j) {
        q.start_d[j] = d.start[j];
        q.goal_d[j] = d.goal[j];
        q.start[j] = (float)d.start[j];
        q.goal[j] = (float)d.goal[j];
    }
    q.w_terminal_d = d.w_terminal;
    q.w_control_d = d.w_control;
    q.w_terminal = (float)d.w_terminal;
    q.w_control = (float)d.w_control;
    q.dt = (float)d.dt;
    q.kappa = (float)d.kappa;
    q.inv_c2 = (float)q.inv_c2_d;
    q.mu = (float)d.mu;
    q.sc_cone = (float)q.sc_cone_d;
    q.K = d.knots_per_segment;
    q.Lmax = d.max_segments;
    q.n_modes = d.n_modes;
    q.task = d.task;
    q.mass_d = d.mass;
    q.ground_mu_d = d.ground_mu;
    q.mass = (float)d.mass;
    q.ground_mu = (float)d.ground_mu;
    const double kth = q.dt_d * q.kappa_d * q.inv_c2_d;
    q.kth_hi = (float)kth;
    q.kth_lo = (float)(kth - (double)q.kth_hi);
    for (int f = 0; f < 4; ++f) q.a_lo[f] = (float)(q.a_d[f] - (double)q.a[f]);
    const double kc = q.kappa_d * q.inv_c2_d;
    q.kc_hi = (float)kc;
    q.kc_lo = (float)(kc - (double)q.kc_hi);
}

// Solver parameters of a call from the options and an iteration budget
// (max_iters <= 0 keeps opts.max_iters).
SolverParams make_params(const comet_solver_opts& o, int max_iters) {
    SolverParams sp;
    memset(&sp, 0, sizeof(sp));
    sp.max_iters = max_iters > 0 ? max_iters : o.max_iters;
    sp.max_retries = 8;
    sp.n_alpha = 7;
    sp.max_inner = 40;
    sp.curv_skip = 3;
    sp.beta0 = (float)o.beta0;
    sp.beta_max = (float)o.beta_max;
    sp.beta_growth = 10.f;
    sp.beta_ref = (float)o.beta_ref;
    sp.rho0 = (float)o.rho0;
    sp.rho_min = (float)o.rho_min;
    sp.rho_max = 1e6f;
    sp.armijo_c1 = 1e-4f;
    sp.ls_slack = 1e-6f;
    sp.eps_primal = (float)o.eps_primal;
    sp.eps_dual = (float)o.eps_dual;
    sp.eps_comp = (float)o.eps_comp;
    sp.omega_ratio = 1.f;
    sp.eta_ratio = 0.25f;
    sp.eps_feas = o.eps_feas;
    sp.merit_mu = o.merit_mu;
    sp.refine = o.precision_flags & 1;
    sp.refine_beta = (float)o.refine_beta;
    return sp;
}

// Validate the instance descriptors; returns COMET_OK and N_max.
comet_status check_instances(const comet_instance_desc* inst, int32_t n_instances, int* Nmax_out);

}  // namespace comet

namespace comet {
// Record a call-level error message for comet_last_error().
void set_error(const char* msg) { g_err = msg; }
}  // namespace comet

namespace comet {
// Options of a call: the defaults, overridden by every positive field of
// `opts` (NULL = defaults); precision_flags is taken as given.
void merge_opts(const comet_solver_opts* opts, comet_solver_opts* out) {
    comet_default_opts(out);
    if (!opts) return;
    const comet_solver_opts& o = *opts;
    if (o.max_iters > 0) out->max_iters = o.max_iters;
    if (o.ref_iters > 0) out->ref_iters = o.ref_iters;
    if (o.eps_feas > 0) out->eps_feas = o.eps_feas;
    if (o.eps_primal > 0) out->eps_primal = o.eps_primal;
    if (o.eps_dual > 0) out->eps_dual = o.eps_dual;
    if (o.eps_comp > 0) out->eps_comp = o.eps_comp;
    if (o.merit_mu > 0) out->merit_mu = o.merit_mu;
    if (o.beta0 > 0) out->beta0 = o.beta0;
    if (o.beta_max > 0) out->beta_max = o.beta_max;
    if (o.beta_ref > 0) out->beta_ref = o.beta_ref;
    if (o.rho0 > 0) out->rho0 = o.rho0;
    if (o.rho_min > 0) out->rho_min = o.rho_min;
    if (o.refine_beta > 0) out->refine_beta = o.refine_beta;
    out->precision_flags = o.precision_flags;
}
}  // namespace comet



namespace comet {
comet_status check_instances(const comet_instance_desc* inst, int32_t n_instances, int* Nmax_out) {
    int Nmax = 0;
    for (int i = 0; i < n_instances; ++i) {
        const comet_instance_desc& d = inst[i];
        if (d.task != COMET_TASK_PUSHER_SLIDER && d.task != COMET_TASK_BIMANUAL)
            return fail(COMET_ERR_INVALID_ARG, "instance %d: unknown task %d", i, d.task);
        if (d.task != inst[0].task) return fail(COMET_ERR_INVALID_ARG, "instance %d: a problem holds one task", i);
        if (d.task == COMET_TASK_PUSHER_SLIDER && d.n_modes != 12 && d.n_modes != 13)
            return fail(COMET_ERR_INVALID_ARG, "instance %d: pushing needs n_modes = 12 or 13 (with free motion)", i);
        // mode codes (base n_modes + 1) stay below 2^64: 13^17 and 14^16 fit
        if (d.task == COMET_TASK_PUSHER_SLIDER && d.n_modes == 13 && d.max_segments > 15)
            return fail(COMET_ERR_INVALID_ARG, "instance %d: with free motion max_segments <= 15", i);
        if (d.task == COMET_TASK_BIMANUAL) {
            if (d.n_modes != 507) return fail(COMET_ERR_INVALID_ARG, "instance %d: bimanual needs n_modes = 507", i);
            if (!(d.mass > 0 && d.ground_mu >= 0 && d.side_x > 0 && d.side_y > 0 && d.dt > 0 && d.mu >= 0))
                return fail(COMET_ERR_INVALID_ARG, "instance %d: bad bimanual geometry, mass or friction", i);
            if (d.max_segments < 1 || d.max_segments > COMET_MAX_SEGMENTS || d.knots_per_segment < 1 ||
                (int64_t)d.knots_per_segment * d.max_segments > 512)
                return fail(COMET_ERR_INVALID_ARG, "instance %d: bad knots_per_segment / max_segments", i);
            Nmax = std::max(Nmax, d.knots_per_segment * d.max_segments);
            continue;
        }
        if (d.knots_per_segment < 1 || d.max_segments < 1 || d.max_segments > COMET_MAX_SEGMENTS ||
            (int64_t)d.knots_per_segment * d.max_segments > comet::kMaxN)
            return fail(COMET_ERR_INVALID_ARG, "instance %d: bad knots_per_segment / max_segments", i);
        if (!(d.side_x > 0 && d.side_y > 0 && d.c_ls > 0 && d.dt > 0 && d.mu >= 0 && d.kappa > 0))
            return fail(COMET_ERR_INVALID_ARG, "instance %d: non-positive geometry or dt", i);
        Nmax = std::max(Nmax, d.knots_per_segment * d.max_segments);
    }
    *Nmax_out = Nmax;
    return COMET_OK;
}
}  // namespace comet

namespace comet {

static int64_t resident_warps(const comet_problem* p, int64_t n) {
    // bimanual: one CTA per TO, the workspace unit is a CTA
    if (p->task == COMET_TASK_BIMANUAL)
        return std::min<int64_t>((int64_t)p->num_sms * p->blocks_per_sm, std::max<int64_t>(n, 1));
    // resident warps: every SM filled, never more warps than TOs; the grid is
    // whole CTAs and any warp may pick any TO, so the workspace covers them all
    const int64_t resident = (int64_t)p->num_sms * p->blocks_per_sm * p->warps_per_block;
    return ((std::min<int64_t>(resident, std::max<int64_t>(n, 1)) + p->warps_per_block - 1) / p->warps_per_block) *
           p->warps_per_block;
}

// floats of workspace per unit (a warp for pushing, a CTA for bimanual)
static int64_t ws_unit_floats(const comet_problem* p) {
    return (int64_t)(p->task == COMET_TASK_BIMANUAL ? kBimRec : kRec) * p->Nmax;
}

comet_status reserve_eval(comet_problem* p, int64_t n) {
    if (p->stats_cap < n) {
        cudaFree(p->d_viol); cudaFree(p->d_merit); cudaFree(p->d_iters); cudaFree(p->d_stat);
        p->d_viol = p->d_merit = p->d_stat = nullptr;
        p->d_iters = nullptr;
        p->stats_cap = 0;
        const int64_t cap = std::max<int64_t>(n, 1024);
        CUDA_TRY(cudaMalloc(&p->d_viol, sizeof(float) * cap), "stats");
        CUDA_TRY(cudaMalloc(&p->d_merit, sizeof(float) * cap), "stats");
        CUDA_TRY(cudaMalloc(&p->d_iters, sizeof(int32_t) * cap), "stats");
        CUDA_TRY(cudaMalloc(&p->d_stat, sizeof(float) * cap), "stats");
        p->stats_cap = cap;
    }
    if (p->hetero && p->perm_cap < n) {
        cudaFree(p->d_perm);
        p->d_perm = nullptr;
        p->perm_cap = 0;
        CUDA_TRY(cudaMalloc(&p->d_perm, sizeof(unsigned int) * std::max<int64_t>(n, 1)), "order buffer");
        p->perm_cap = n;
        if (!p->d_lpt) CUDA_TRY(cudaMalloc(&p->d_lpt, lpt_scratch_bytes()), "order scratch");
    }
    const int64_t warps = resident_warps(p, n);
    if (p->ws_warps < warps) {
        cudaFree(p->d_ws);
        p->d_ws = nullptr;
        p->ws_warps = 0;
        CUDA_TRY(cudaMalloc(&p->d_ws, sizeof(float) * (size_t)ws_unit_floats(p) * warps), "workspace");
        p->ws_warps = warps;
    }
    return COMET_OK;
}

comet_status launch_eval_device(comet_problem* p, const comet_mode_seq* d_seqs, int64_t n_max, const int64_t* d_n,
                                const float* d_warm, int32_t max_iters, float* d_cost, float* d_traj,
                                int32_t* d_status) {
    cudaStream_t s = p->stream;
    const int64_t warps = resident_warps(p, n_max);
    if (p->ws_warps < warps || p->stats_cap < n_max) return fail(COMET_ERR_INTERNAL, "evaluator not reserved");
    CUDA_TRY(cudaMemsetAsync(p->d_queue, 0, sizeof(unsigned int), s), "queue reset");
    CUDA_TRY(cudaMemsetAsync(p->d_bad, 0, sizeof(int), s), "flag reset");
    // mixed interval counts: hand the TOs out longest first
    const bool lpt = p->hetero && p->perm_cap >= n_max && n_max > 1;
    if (lpt)
        CUDA_TRY(launch_lpt_order(d_seqs, n_max, d_n, p->d_inst, (int)p->inst.size(), p->d_lpt, p->d_perm, s),
                 "longest-first order");
    EvalArgs a;
    memset(&a, 0, sizeof(a));
    a.inst = p->d_inst;
    a.n_inst = (int)p->inst.size();
    a.seqs = d_seqs;
    a.n = n_max;
    a.d_n = d_n;
    a.perm = lpt ? p->d_perm : nullptr;
    a.warm = d_warm;
    a.stride = p->stride;
    a.Nmax = p->Nmax;
    a.out_cost = d_cost;
    a.out_traj = d_traj;
    a.out_status = d_status;
    a.out_viol = p->d_viol;
    a.out_merit = p->d_merit;
    a.out_iters = p->d_iters;
    a.out_stat = p->d_stat;
    a.ws = p->d_ws;
    a.ws_per_warp = ws_unit_floats(p);
    a.queue = p->d_queue;
    a.bad_input = p->d_bad;
    a.unroll = p->unroll;
    a.stall_staging = p->stall_staging;
    a.sp = make_params(p->opts, max_iters);
    for (const comet_instance_desc& d : p->inst) a.sp.free_motion |= d.task == COMET_TASK_PUSHER_SLIDER && d.n_modes == 13;
    if (p->task == COMET_TASK_BIMANUAL)
        CUDA_TRY(launch_bimanual(a, (int)warps, s), "bimanual evaluator launch");
    else
        CUDA_TRY(launch_eval(a, (int)warps, p->warps_per_block, s), "evaluator launch");
    return COMET_OK;
}

}  // namespace comet

extern "C" {

comet_status comet_default_opts(comet_solver_opts* o) {
    if (!o) return fail(COMET_ERR_INVALID_ARG, "opts is NULL");
    memset(o, 0, sizeof(*o));
    o->max_iters = 300;
    o->ref_iters = 1500;
    o->eps_feas = 1e-5;
    o->eps_primal = 1e-6;
    o->eps_dual = 1e-4;
    o->eps_comp = 1e-6;
    o->merit_mu = 100.0;
    o->beta0 = 100.0;
    o->beta_max = 1e4;
    o->beta_ref = 1e3;
    o->rho0 = 1e-4;
    o->rho_min = 1e-4;
    o->precision_flags = 1;
    o->refine_beta = 1e4;
    return COMET_OK;
}

const char* comet_last_error(void) { return g_err.c_str(); }

uint64_t comet_mode_code(const comet_mode_seq* seq, int32_t n_modes) {
    if (!seq || n_modes < 1 || seq->len < 1 || seq->len > COMET_MAX_SEGMENTS) return 0;
    const unsigned __int128 base = (unsigned __int128)(n_modes + 1);
    unsigned __int128 code = seq->len, p = base;
    for (int i = 0; i < seq->len; ++i) {
        if (seq->modes[i] >= n_modes) return 0;
        code += (unsigned __int128)(seq->modes[i] + 1) * p;
        p *= base;
    }
    if (code >> 64) return 0;
    return (uint64_t)code;
}

int64_t comet_traj_stride(const comet_problem* p) { return p ? p->stride : 0; }

comet_status comet_problem_create(const comet_instance_desc* inst, int32_t n_instances,
                                  const comet_solver_opts* opts, void* cuda_stream, comet_problem** out) {
    if (!out) return fail(COMET_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!inst || n_instances < 1) return fail(COMET_ERR_INVALID_ARG, "need at least one instance");
    int Nmax = 0;
    {
        const comet_status st = comet::check_instances(inst, n_instances, &Nmax);
        if (st != COMET_OK) return st;
    }
    comet_problem* p = new (std::nothrow) comet_problem();
    if (!p) return fail(COMET_ERR_OOM, "host allocation failed");
    comet::merge_opts(opts, &p->opts);
    p->inst.assign(inst, inst + n_instances);
    for (int i = 0; i < n_instances; ++i)
        if (inst[i].max_segments > 1 || inst[i].knots_per_segment != inst[0].knots_per_segment) p->hetero = true;
    p->stream = (cudaStream_t)cuda_stream;
    p->Nmax = Nmax;
    p->task = inst[0].task;
    p->stride = p->task == COMET_TASK_BIMANUAL ? 17 * (int64_t)Nmax + 5 : 7 * (int64_t)Nmax + 4;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "device query");
    }
    std::vector<comet::DevInstance> h(n_instances);
    for (int i = 0; i < n_instances; ++i) comet::make_dev_instance(inst[i], &h[i]);
    e = cudaMalloc(&p->d_inst, sizeof(comet::DevInstance) * n_instances);
    if (e == cudaSuccess) e = cudaMemcpy(p->d_inst, h.data(), sizeof(comet::DevInstance) * n_instances,
                                         cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_queue, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&p->d_bad, sizeof(int));
    if (e != cudaSuccess) {
        comet_problem_destroy(p);
        return cuda_fail(e, "problem allocation");
    }
    const size_t smem = comet::smem_per_warp_bytes(Nmax) * p->warps_per_block;
    if (p->task == COMET_TASK_BIMANUAL) {
        p->warps_per_block = comet::kBimThreads / 32;
        p->blocks_per_sm = comet::bim_blocks_per_sm(Nmax);
        if (p->blocks_per_sm < 1) {
            comet_problem_destroy(p);
            return fail(COMET_ERR_INVALID_ARG, "N_max = %d does not fit the bimanual evaluator", Nmax);
        }
        *out = p;
        return COMET_OK;
    }
    p->blocks_per_sm = comet::eval_blocks_per_sm(p->warps_per_block, smem);
    {
        // a shape the autotuner picked for this device and N_max
        int w = 0, b = 0, un = 1;
        if (p->blocks_per_sm >= 1 && comet::cached_launch_shape(p->device, Nmax, &w, &b, &un)) {
            const int occ = comet::eval_blocks_per_sm(w, comet::smem_per_warp_bytes(Nmax) * w);
            if (occ >= b && b >= 1) {
                p->warps_per_block = w;
                p->blocks_per_sm = b;
                p->unroll = un;
            }
        }
    }
    if (p->blocks_per_sm < 1) {
        comet_problem_destroy(p);
        return fail(COMET_ERR_INVALID_ARG, "N_max = %d needs %zu bytes of shared memory per block", Nmax, smem);
    }
    *out = p;
    return COMET_OK;
}

comet_status comet_problem_destroy(comet_problem* p) {
    if (!p) return COMET_OK;
    if (p->stream) cudaStreamSynchronize(p->stream); else cudaDeviceSynchronize();
    cudaFree(p->d_inst);
    cudaFree(p->d_queue);
    cudaFree(p->d_bad);
    cudaFree(p->d_ws);
    cudaFree(p->d_tws);
    cudaFree(p->d_viol);
    cudaFree(p->d_merit);
    cudaFree(p->d_iters);
    cudaFree(p->d_stat);
    cudaFree(p->d_stage);
    cudaFree(p->d_perm);
    cudaFree(p->d_lpt);
    delete p;
    return COMET_OK;
}

static comet_status ensure(void** buf, size_t* cap, size_t bytes, const char* what) {
    if (*cap >= bytes) return COMET_OK;
    cudaFree(*buf);
    *buf = nullptr;
    *cap = 0;
    cudaError_t e = cudaMalloc(buf, bytes);
    if (e != cudaSuccess) return cuda_fail(e, what);
    *cap = bytes;
    return COMET_OK;
}

comet_status comet_eval_modes_budget(comet_problem* p, const comet_mode_seq* seqs, int64_t n,
                                     const float* warm, int32_t max_iters, float* out_cost, float* out_traj,
                                     int32_t* out_status) {
    if (!p) return fail(COMET_ERR_INVALID_ARG, "problem is NULL");
    if (n < 0) return fail(COMET_ERR_INVALID_ARG, "n < 0");
    if (n > 0 && (!seqs || !out_cost || !out_status))
        return fail(COMET_ERR_INVALID_ARG, "mode_seqs, out_cost and out_status are required");
    if (max_iters < 0) return fail(COMET_ERR_INVALID_ARG, "max_iters < 0");
    if (n > 0xffffffffLL) return fail(COMET_ERR_INVALID_ARG, "n too large");
    CUDA_TRY(cudaSetDevice(p->device), "cudaSetDevice");
    cudaStream_t s = p->stream;
    {
        const comet_status st = comet::reserve_eval(p, n);
        if (st != COMET_OK) return st;
    }
    p->last_n = n;
    if (n == 0) return COMET_OK;

    const bool dev_seqs = is_device_ptr(seqs);
    const bool dev_warm = warm ? is_device_ptr(warm) : true;
    const bool dev_cost = is_device_ptr(out_cost);
    const bool dev_traj = out_traj ? is_device_ptr(out_traj) : true;
    const bool dev_status = is_device_ptr(out_status);
    const size_t traj_bytes = sizeof(float) * (size_t)p->stride * (size_t)n;
    if (!dev_seqs) {
        // validate host orders before any work
        for (int64_t i = 0; i < n; ++i) {
            const comet_mode_seq& q = seqs[i];
            if (q.instance < 0 || q.instance >= (int)p->inst.size())
                return fail(COMET_ERR_INVALID_ARG, "order %lld: instance %d out of range", (long long)i, q.instance);
            const comet_instance_desc& d = p->inst[q.instance];
            if (q.len < 1 || q.len > d.max_segments)
                return fail(COMET_ERR_INVALID_ARG, "order %lld: length %d out of range", (long long)i, q.len);
            for (int j = 0; j < q.len; ++j)
                if (q.modes[j] >= d.n_modes)
                    return fail(COMET_ERR_INVALID_ARG, "order %lld: mode %d out of range", (long long)i, q.modes[j]);
        }
    }
    // staging layout: seqs | warm | cost | status | traj
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_seqs = dev_seqs ? 0 : take(sizeof(comet_mode_seq) * n);
    const size_t o_warm = dev_warm ? 0 : take(traj_bytes);
    const size_t o_cost = dev_cost ? 0 : take(sizeof(float) * n);
    const size_t o_status = dev_status ? 0 : take(sizeof(int32_t) * n);
    const size_t o_traj = dev_traj ? 0 : take(traj_bytes);
    if (off) {
        comet_status st = ensure(&p->d_stage, &p->stage_bytes, off, "staging buffer");
        if (st != COMET_OK) return st;
    }
    char* stage = (char*)p->d_stage;
    const comet_mode_seq* d_seqs = seqs;
    const float* d_warm = warm;
    float* d_cost = out_cost;
    int32_t* d_status = out_status;
    float* d_traj = out_traj;
    if (!dev_seqs) {
        d_seqs = (const comet_mode_seq*)(stage + o_seqs);
        CUDA_TRY(cudaMemcpyAsync((void*)d_seqs, seqs, sizeof(comet_mode_seq) * n, cudaMemcpyHostToDevice, s),
                 "copy orders");
    }
    if (!dev_warm) {
        d_warm = (const float*)(stage + o_warm);
        CUDA_TRY(cudaMemcpyAsync((void*)d_warm, warm, traj_bytes, cudaMemcpyHostToDevice, s), "copy warm starts");
    }
    if (!dev_cost) d_cost = (float*)(stage + o_cost);
    if (!dev_status) d_status = (int32_t*)(stage + o_status);
    if (!dev_traj) d_traj = (float*)(stage + o_traj);

    {
        const comet_status st =
            comet::launch_eval_device(p, d_seqs, n, nullptr, d_warm, max_iters, d_cost, d_traj, d_status);
        if (st != COMET_OK) return st;
    }

    if (!dev_cost) CUDA_TRY(cudaMemcpyAsync(out_cost, d_cost, sizeof(float) * n, cudaMemcpyDeviceToHost, s), "copy cost");
    if (!dev_status)
        CUDA_TRY(cudaMemcpyAsync(out_status, d_status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s), "copy status");
    if (!dev_traj) CUDA_TRY(cudaMemcpyAsync(out_traj, d_traj, traj_bytes, cudaMemcpyDeviceToHost, s), "copy traj");
    if (!(dev_seqs && dev_warm && dev_cost && dev_status && dev_traj)) {
        CUDA_TRY(cudaStreamSynchronize(s), "synchronise");
        int flag = 0;
        CUDA_TRY(cudaMemcpy(&flag, p->d_bad, sizeof(int), cudaMemcpyDeviceToHost), "read the device flag");
        if (flag == 2) return fail(COMET_ERR_TIMEOUT, "a bounded device wait ran out (warm-start staging)");
    }
    return COMET_OK;
}

comet_status comet_eval_check(comet_problem* p, int32_t* out_flag) {
    if (!p) return fail(COMET_ERR_INVALID_ARG, "problem is NULL");
    CUDA_TRY(cudaSetDevice(p->device), "cudaSetDevice");
    CUDA_TRY(cudaStreamSynchronize(p->stream), "synchronise");
    int flag = 0;
    CUDA_TRY(cudaMemcpy(&flag, p->d_bad, sizeof(int), cudaMemcpyDeviceToHost), "read the device flag");
    if (out_flag) *out_flag = flag;
    if (flag == 2) return fail(COMET_ERR_TIMEOUT, "a bounded device wait ran out (warm-start staging)");
    return COMET_OK;
}

comet_status comet_debug_stall_staging(comet_problem* p, int32_t on) {
    if (!p) return fail(COMET_ERR_INVALID_ARG, "problem is NULL");
    p->stall_staging = on ? 1 : 0;
    return COMET_OK;
}

comet_status comet_eval_modes(comet_problem* p, const comet_mode_seq* seqs, int64_t n, const float* warm,
                              float* out_cost, float* out_traj, int32_t* out_status) {
    return comet_eval_modes_budget(p, seqs, n, warm, 0, out_cost, out_traj, out_status);
}

comet_status comet_eval_modes_timed(comet_problem* p, const comet_timing_opts* timing,
                                    const comet_mode_seq* mode_seqs, int64_t n, const float* warm_starts,
                                    int32_t max_iters, float* out_cost, float* out_traj, int32_t* out_status) {
    if (!p || !timing) return fail(COMET_ERR_INVALID_ARG, "problem and timing are required");
    if (p->task != COMET_TASK_PUSHER_SLIDER)
        return fail(COMET_ERR_INVALID_ARG, "timing optimisation is defined for pushing problems");
    if (!(timing->h_min > 0.0 && timing->h_min <= timing->h_max && timing->T_max > 0.0))
        return fail(COMET_ERR_INVALID_ARG, "timing bounds: need 0 < h_min <= h_max and T_max > 0");
    if (n < 0 || n > 0xffffffffLL) return fail(COMET_ERR_INVALID_ARG, "n out of range");
    if (max_iters < 0) return fail(COMET_ERR_INVALID_ARG, "max_iters < 0");
    if (n == 0) {
        p->last_n = 0;
        return COMET_OK;
    }
    if (!mode_seqs || !out_cost || !out_status)
        return fail(COMET_ERR_INVALID_ARG, "mode_seqs, out_cost and out_status are required");
    if (!is_device_ptr(mode_seqs) || !is_device_ptr(out_cost) || !is_device_ptr(out_status) ||
        (warm_starts && !is_device_ptr(warm_starts)) || (out_traj && !is_device_ptr(out_traj)))
        return fail(COMET_ERR_INVALID_ARG, "comet_eval_modes_timed takes device arrays only");
    CUDA_TRY(cudaSetDevice(p->device), "cudaSetDevice");
    int smem_optin = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device),
             "shared memory limit");
    const size_t per_warp = comet::timing_smem_per_warp_bytes(p->Nmax);
    int wpb = 4;
    while (wpb > 1 && per_warp * wpb > (size_t)smem_optin) --wpb;
    if (per_warp * wpb > (size_t)smem_optin)
        return fail(COMET_ERR_INVALID_ARG, "N_max = %d does not fit the timing kernel's shared memory", p->Nmax);
    {
        const comet_status st = comet::reserve_eval(p, n);
        if (st != COMET_OK) return st;
    }
    const int bps = comet::timing_blocks_per_sm(wpb, p->Nmax);
    if (bps < 1) return fail(COMET_ERR_CUDA, "timing kernel: no resident block");
    const int64_t resident = (int64_t)p->num_sms * bps * wpb;
    const int64_t warps = ((std::min<int64_t>(resident, n) + wpb - 1) / wpb) * wpb;
    const int64_t ws_floats = comet::timing_ws_per_warp_floats(p->Nmax) * warps;
    if (p->tws_floats < ws_floats) {
        cudaFree(p->d_tws);
        p->d_tws = nullptr;
        p->tws_floats = 0;
        CUDA_TRY(cudaMalloc(&p->d_tws, sizeof(float) * (size_t)ws_floats), "timing workspace");
        p->tws_floats = ws_floats;
    }
    cudaStream_t s = p->stream;
    CUDA_TRY(cudaMemsetAsync(p->d_queue, 0, sizeof(unsigned int), s), "queue reset");
    CUDA_TRY(cudaMemsetAsync(p->d_bad, 0, sizeof(int), s), "flag reset");
    comet::TimingArgs a;
    memset(&a, 0, sizeof(a));
    a.e.inst = p->d_inst;
    a.e.n_inst = (int)p->inst.size();
    a.e.seqs = mode_seqs;
    a.e.n = n;
    a.e.warm = warm_starts;
    a.e.stride = 9 * (int64_t)p->Nmax + 5;
    a.e.Nmax = p->Nmax;
    a.e.out_cost = out_cost;
    a.e.out_traj = out_traj;
    a.e.out_status = out_status;
    a.e.out_viol = p->d_viol;
    a.e.out_merit = p->d_merit;
    a.e.out_iters = p->d_iters;
    a.e.out_stat = p->d_stat;
    a.e.ws = p->d_tws;
    a.e.ws_per_warp = comet::timing_ws_per_warp_floats(p->Nmax);
    a.e.queue = p->d_queue;
    a.e.bad_input = p->d_bad;
    a.e.sp = comet::make_params(p->opts, max_iters);
    a.h_min = (float)timing->h_min;
    a.h_max = (float)timing->h_max;
    a.T = (float)timing->T_max;
    p->last_n = n;
    CUDA_TRY(comet::launch_timing(a, (int)warps, wpb, s), "timing kernel launch");
    return COMET_OK;
}

comet_status comet_eval_stats(comet_problem* p, float* out_viol, float* out_merit, int32_t* out_iters,
                              float* out_stat) {
    if (!p) return fail(COMET_ERR_INVALID_ARG, "problem is NULL");
    const int64_t n = p->last_n;
    if (n == 0) return COMET_OK;
    cudaStream_t s = p->stream;
    bool host = false;
    struct Item {
        void* dst;
        const void* src;
        size_t bytes;
    } items[4] = {{out_viol, p->d_viol, sizeof(float) * n},
                  {out_merit, p->d_merit, sizeof(float) * n},
                  {out_iters, p->d_iters, sizeof(int32_t) * n},
                  {out_stat, p->d_stat, sizeof(float) * n}};
    for (auto& it : items) {
        if (!it.dst) continue;
        const bool dev = is_device_ptr(it.dst);
        host = host || !dev;
        CUDA_TRY(cudaMemcpyAsync(it.dst, it.src, it.bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s),
                 "copy stats");
    }
    if (host) CUDA_TRY(cudaStreamSynchronize(s), "synchronise");
    return COMET_OK;
}

}  // extern "C"
