// state.h -- plain-old-data layouts shared by host and device code.
#pragma once
#include <stdint.h>

namespace pdcs {

// Scalars of Algorithm 1 kept in device memory.  Every per-iteration decision
// (step acceptance, Halpern coefficients, restart, primal weight, termination)
// is taken by a device thread; the host only reads `status` between chunks.
struct Ctrl {
    // PDHG step (eq. PDHG): tau = eta / omega, sigma = eta * omega
    double eta, omega, tau, sigma;
    // pending ReflectedHalpern update of the last accepted evaluation:
    // z <- ha * zhat + hb * z + hc * z0, then zsum += hw * z
    double ha, hb, hc, hw;
    double wsum;          // sum of average weights since the last restart
    double beta;          // reflection parameter
    double tol;           // termination tolerance (<= 0: off)
    double phi0;          // restart metric of the current anchor z^{t,0}
    double phi_prev;      // restart metric of the previous check's candidate
    double comp0[3];      // ||r_p||^2, ||r_d||^2, gap of the anchor (to re-weight phi)
    double err[3];        // relative errors of the returned solution
    double pobj, dobj;    // its objective values
    double hmax, cmax;    // ||h||_inf, ||c||_inf of the original data
    long long attempts;   // PDHG evaluations so far
    long long accepted;   // accepted steps so far
    long long k;          // accepted steps since the last restart
    long long restarts;
    int32_t pending;      // 1: the Halpern update of the last evaluation is not applied yet
    int32_t status;       // kRunning / kConverged / kNumericError / kTimeout
    int32_t step_mode;    // 0 adaptive, 1 constant, 2 plain
    int32_t check_mode;   // 0 regular check, 1 initial evaluation of the anchor
    int32_t restart_now;  // set by the check controller: 1 restart to candidate `best`
    int32_t best;         // candidate chosen by the last check (0 current, 1 average)
    int32_t sol_cand;     // candidate copied into the solution by the last check
    int32_t n_cand;       // candidates evaluated by the last check (1 or 2)
    unsigned int ticket;  // block counter of the last-block reductions
    int32_t team_abort;   // set when a bounded wait of the grid-wise SOC projection gave up
    // x-hat buffers (fused K' product + primal update, see spmv_kt_primal): xsel names the
    // buffer holding the x-hat of the current / last evaluation; xnext = 1 when the next
    // evaluation's x-hat (and the accepted step's update of x, K'y, xsum) was already formed,
    // in the other buffer, by the K' product's epilogue
    int32_t xsel, xnext;
};

// Fixed slots of the partial-sum buffer (one double per block per quantity).
// Every kernel that reduces writes its per-block partials to its own region,
// and the consumer adds them in block order, so all sums are deterministic.
struct PartLayout {
    int primal_blocks;  // blocks of the primal update (||dx||^2)
    int dual_blocks;    // blocks of the dual update (||dy||^2, dy'K dx)
    int kktp_blocks;    // blocks of the primal-side KKT kernel, per candidate
    int kktd_blocks;    // blocks of the dual-side KKT kernel, per candidate
    // offsets into the partial buffer
    long long off_px, off_dy, off_kp, off_kd;
    long long total;
};

// quantities of the primal-side KKT kernel (per candidate): rows of K
enum KktP { kpRp2 = 0, kpHy, kpDy2, kpRmax, kpKxmax, kpPmax, kKktPN };
// quantities of the dual-side KKT kernel (per candidate): columns of K
enum KktD { kdRd2 = 0, kdPobj, kdBterm, kdDx2, kdDmax, kdKtymax, kKktDN };

}  // namespace pdcs
