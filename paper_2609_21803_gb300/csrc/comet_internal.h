// comet_internal.h -- types shared by the CUDA translation units of the
// library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "comet.h"

namespace comet {

// Floats per stage record in the per-warp workspace: the u-block Cholesky
// factor and coupling (33), the reduced (y, x, rhs) matrix (44), padded.
constexpr int kRec = 80;
// Largest number of intervals of one TO.
constexpr int kMaxN = 4096;

// FP32 (and FP64 for the certificate) constants of one instance.
struct DevInstance {
    float dt, kappa, inv_c2, mu, sc_cone;  // sc_cone = 1/sqrt(1+mu^2)
    float inv_sigma[4];                    // dynamics-row scaling 1/sigma_r
    float a[4], ell[4];                    // half-depth / half-length of face f
    float start[3], goal[3];
    float w_terminal, w_control;
    int32_t K, Lmax, n_modes, task;
    float mass, ground_mu;               // bimanual: box mass, ground friction
    double dt_d, kappa_d, inv_c2_d, mu_d, sc_cone_d;
    double sigma_d[4];
    double a_d[4], ell_d[4];
    double start_d[3], goal_d[3];
    double w_terminal_d, w_control_d;
    double mass_d, ground_mu_d;
    // theta-row gain K = dt kappa / c^2 as an FP32 pair (hi + lo) and the
    // FP32 rounding residues of the face half-depths, for the theta defect
    // evaluated in double-float
    float kth_hi, kth_lo;
    float a_lo[4];
    // kappa / c^2 as an FP32 pair, for the theta row with a variable
    // interval duration (timing optimisation)
    float kc_hi, kc_lo;
};

struct SolverParams {
    int max_iters, max_retries, n_alpha, max_inner, curv_skip;
    float beta0, beta_max, beta_growth, beta_ref;
    float rho0, rho_min, rho_max;
    float armijo_c1, ls_slack;
    float eps_primal, eps_dual, eps_comp, omega_ratio, eta_ratio;
    double eps_feas, merit_mu;
    int refine;          // FP64 iterative refinement of the step ...
    float refine_beta;   // ... while the penalty exceeds this value
    int free_motion;     // some instance has the free-motion mode (13 pushing modes)
};

struct EvalArgs {
    const DevInstance* inst;
    int n_inst;
    const comet_mode_seq* seqs;
    int64_t n;               // number of TOs (upper bound when d_n is set)
    const int64_t* d_n;      // optional device-resident TO count
    const unsigned int* perm;  // optional order in which warps take the TOs
    const float* warm;
    int64_t stride;  // floats per trajectory record (7*Nmax+4)
    int Nmax;
    float* out_cost;
    float* out_traj;
    int32_t* out_status;
    float* out_viol;
    float* out_merit;
    int32_t* out_iters;
    float* out_stat;
    float* ws;               // per-warp stage records
    int64_t ws_per_warp;     // floats
    unsigned int* queue;     // work counter (next TO index)
    int* bad_input;          // set when a malformed order is met
    int unroll;              // stages per trip of the stage loops (1 or 2)
    int stall_staging;       // test hook: warm-start staging copies are not issued, so
                             // the bounded wait on them runs out (never in a release call)
    SolverParams sp;
};

// Host-side conversions shared by the entry points (api.cu).
void make_dev_instance(const comet_instance_desc& d, DevInstance* out);
SolverParams make_params(const comet_solver_opts& o, int max_iters);
comet_status check_instances(const comet_instance_desc* inst, int32_t n_instances, int* Nmax_out);
void merge_opts(const comet_solver_opts* opts, comet_solver_opts* out);
void set_error(const char* msg);

// Bimanual variant (bimanual_kernel.cu): one CTA of kBimThreads threads per
// TO; per-CTA workspace kBimRec floats per stage.
constexpr int kBimRec = 328;
constexpr int kBimThreads = 128;
size_t bim_smem_bytes(int Nmax);
int bim_blocks_per_sm(int Nmax);
cudaError_t launch_bimanual(const EvalArgs& a, int n_ctas, cudaStream_t s);

// Timing optimisation of the pushing TO (timing_kernel.cu): the arguments
// of the evaluator plus the duration bounds; per-warp workspace of
// timing_ws_per_warp_floats(N_max) floats.
struct TimingArgs {
    EvalArgs e;
    float h_min, h_max, T;
};
size_t timing_smem_per_warp_bytes(int Nmax);
int64_t timing_ws_per_warp_floats(int Nmax);
int timing_blocks_per_sm(int warps_per_block, int Nmax);
cudaError_t launch_timing(const TimingArgs& a, int total_warps, int warps_per_block, cudaStream_t s);

// Launch shape cached by the autotuner for (device, N_max) (autotune.cu).
bool cached_launch_shape(int device, int nmax, int* wpb, int* bps, int* unroll);

// Longest-first order of a batch (schedule.cu): perm[0..n) lists the TOs by
// decreasing interval count; scratch holds lpt_scratch_bytes().
size_t lpt_scratch_bytes();
cudaError_t launch_lpt_order(const comet_mode_seq* seqs, int64_t n, const int64_t* d_n, const DevInstance* inst,
                             int n_inst, unsigned int* scratch, unsigned int* perm, cudaStream_t s);

// Shared memory (bytes) one warp needs for TOs of up to Nmax intervals.
size_t smem_per_warp_bytes(int Nmax);
// Launch the persistent evaluator: total_warps warps, warps_per_block per CTA.
cudaError_t launch_eval(const EvalArgs& a, int total_warps, int warps_per_block, cudaStream_t s);
// Occupancy of the evaluator for the given per-warp shared memory.
int eval_blocks_per_sm(int warps_per_block, size_t smem_per_block);

}  // namespace comet
