// Internal interfaces between the solver, the Lanczos routines and the map.
#pragma once

#include <vector>

#include "kernels.cuh"

namespace msb {

constexpr int kMaxShifts = 4096;

// Per-shift device arrays of the multi-shift recurrence.
struct ShiftArrays {
    double2* zeta;        // zeta^k_m
    double2* zeta_prev;   // zeta^k_{m-1}
    double2* shift;       // s_k
    double2* coef64;      // [k][B][2]: (gamma, c) of each iteration of the block, FP64
    void* coefv;          // same in the vector precision (double2 or float2)
    int* active;          // 1 while the shift iterates
    int* conv;            // 1 once it met the tolerance
    int* broken;          // 1 if zeta_{m+1} = 0 stopped it
    int* nblk;            // iterations of the current block to apply
    int* iters;           // iteration at freeze
    double* resid;        // ||r_m|| / (|zeta_m| ||b||) at freeze
    int* zexp;            // E_k = log2(g_k / S_m): exponent of the stored zeta pair
    double2* fz_coef;     // r^k_m = fz_coef * (stored r~_m) for the shift's latest residual
    int* fz_iter;         // the iteration m of that residual (Eq. 4 at freeze, or at the end)
};

struct SolveProblem {
    int64_t n = 0;            // seed dimension
    int ns = 0;               // shifts
    const void* b = nullptr;  // device RHS (precision of prec)
    void* x = nullptr;        // device output, ns x n_out
    int64_t n_out = 0;        // per-shift vector length (n, or the projected length)
    const int32_t* rows = nullptr;   // optional row map for the projected output
    int64_t rowlen = 1;
    void* rrec = nullptr;     // optional device output, ns x n_out: each shift's recursive
                              // residual r_m / zeta_m^k (Eq. 4) at its freeze or at the end
    double2 c0{0, 0};
    std::vector<double2> shifts;
    double tol = 1e-10;
    int maxit = 1000;
    int block = 4;
    msb_precision prec = MSB_FP64;
    bool dual = false;        // dual-space BiCG (App. A): A + c0 with A Hermitian, not complex symmetric
};

struct SolveResult {
    int iterations = 0;
    int n_converged = 0;
    int64_t flushes = 0;
    int64_t launches = 0;
    double seed_residual = 0, bnorm = 0;
    std::vector<int> iters, conv;
    std::vector<double> resid;
    msb_status status = MSB_OK;
};

void multishift_solve(msb_op* op, const SolveProblem& pr, SolveResult& out, cudaStream_t st);
// Lag B of the fused per-shift update: `block` if set, else the autotuned choice
// for (n, ns, prec) if there is one (autotune.cu), else 4 (FP64) / 8 (FP32).
int pick_block(int block, msb_precision prec, int64_t n = 0, int ns = 0);
// Autotuned choices (0: none cached).
int tuned_block(int64_t n, int ns, msb_precision prec);
int tuned_cf_threads(int64_t Ddn, int64_t Dup, msb_precision prec);

// Ground state by Lanczos (FP64, real vectors).
struct GroundResult {
    double E = 0, residual = 0;
    int restarts = 0;
    int64_t matvecs = 0;
    int64_t launches = 0;
    msb_status status = MSB_OK;
};
void ground_state(msb_op* H, double tol, int maxit, const double* start, double* g, GroundResult& out,
                  cudaStream_t st);

// Batched Lanczos continued fraction over n_vec columns.
struct CFResult {
    std::vector<int> depth;
    int64_t matvecs = 0;
    int64_t launches = 0;
};
void continued_fraction(msb_op* H, const void* phi, int n_vec, double E0, const double* w, int n_w,
                        double eta, double cf_tol, int cf_check, int cf_maxdepth, msb_precision prec,
                        double* I_out, CFResult& out, cudaStream_t st, bool I_on_device = false);

// Columns of one continued-fraction run.  Column c starts at phi + c * ldphi
// (elements), has ops[q[c]]->dim elements and applies ops[q[c]] with the energy
// origin E0[c]: one operator for all columns, or, for a batch of clusters, each
// column its own cluster's Hubbard H (one launch per step covers all columns).
struct CFColumns {
    const void* phi = nullptr;
    int64_t ldphi = 0;
    int nv = 0;
    std::vector<const msb_op*> ops;
    std::vector<int> q;
    std::vector<double> E0;
};

// The batch form: Hubbard operators only; I_out on the host (nv x n_w).
void continued_fraction_columns(const CFColumns& P, const double* w, int n_w, double eta, double cf_tol,
                                int cf_check, int cf_maxdepth, msb_precision prec, double* I_out, CFResult& out,
                                cudaStream_t st);

// Work runs on an internal non-blocking stream ordered after the caller's
// stream; finish() orders the caller's stream after it and synchronises.
struct StreamScope {
    cudaStream_t user, s;
    cudaEvent_t ev;
    explicit StreamScope(cudaStream_t u) : user(u) {
        MSB_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
        MSB_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        MSB_CUDA(cudaEventRecord(ev, user));
        MSB_CUDA(cudaStreamWaitEvent(s, ev, 0));
    }
    void finish() {
        MSB_CUDA(cudaEventRecord(ev, s));
        MSB_CUDA(cudaStreamWaitEvent(user, ev, 0));
        MSB_CUDA(cudaStreamSynchronize(s));
    }
    ~StreamScope() {
        cudaStreamSynchronize(s);
        cudaEventDestroy(ev);
        cudaStreamDestroy(s);
    }
};

void set_error_message(const std::string& m);

}  // namespace msb
