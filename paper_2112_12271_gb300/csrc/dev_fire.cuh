// dev_fire.cuh -- the FIRE 2.0 scalar update (Guenole et al., Comput. Mater.
// Sci. 175, 109584 (2020); Sec. II.B of the paper names the method), run by one
// thread after the force reduction of an iteration.  fs holds the state and
// parameters (FireSlot indices), red the reduced sums (Red indices) of the
// forces and velocities at the current positions.  The steps are those of the
// published FIRE 2.0 algorithm (its Algorithm 2): on P <= 0, dt *= f_dec
// only while f_dec dt >= dt_min, and the velocity mixing belongs to the MD
// integration step of every iteration.  Order of tests: converged
// (max_i |F_i| < f_tol; or the paper's criteria of Sec. II.B when set:
// E_pair/N < e_thres, or the fractional drop below f_thres ten iterations
// in a row), precision switch, max_iter; then the P = F.v rules.
// The precision switch (FP32 -> FP64 pair forces) happens below the switch
// threshold, or when the FP32 phase stalls (n_neg_max P <= 0 steps in a row).
// Writes and returns the new status.
#pragma once
#include "common.cuh"

namespace hdmd {

__device__ __forceinline__ int fire_scalar_update(double *fs, const double *red) {
    const double fmx = sqrt(red[R_FMAX2]);
    fs[FS_FMAX] = fmx;
    const double E = 0.5 * red[R_E];
    fs[FS_E] = E;
    // the paper's fractional drop |(E_{i+1} - E_i)/E_i| (Eq. (6)), counted
    // once per iteration (a precision switch re-evaluates the same one)
    if (fs[FP_FTHRES] > 0.0 && fs[FS_ITER] != fs[FS_FITER]) {
        const double Ep = fs[FS_EPREV];
        const bool flat = fs[FS_ITER] > 0.0 && Ep != 0.0 && fabs((E - Ep) / Ep) < fs[FP_FTHRES];
        fs[FS_NFLAT] = flat ? fs[FS_NFLAT] + 1.0 : 0.0;
        fs[FS_EPREV] = E;
        fs[FS_FITER] = fs[FS_ITER];
    }
    int status = FIRE_RUNNING;
    if (red[R_BAD] != 0.0) status = FIRE_NEGFAIL;
    else if (fmx < fs[FP_FTOL]) status = FIRE_CONVERGED;
    else if (fs[FP_ETHRES] > 0.0 && E / fs[FP_NATOMS] < fs[FP_ETHRES]) status = FIRE_CONVERGED;
    else if (fs[FP_FTHRES] > 0.0 && fs[FS_NFLAT] >= 10.0) status = FIRE_CONVERGED;
    else if (fmx < fs[FP_SWITCH]) status = FIRE_SWITCH;
    else if (fs[FS_ITER] >= fs[FP_MAXITER]) status = FIRE_MAXITER;
    else {
        double dt = fs[FS_DT], alpha = fs[FS_ALPHA];
        const double P = red[R_P];
        if (P > 0.0) {
            fs[FS_NPOS] += 1.0;
            fs[FS_NNEG] = 0.0;
            if (fs[FS_NPOS] > fs[FP_NDELAY]) {
                dt = fmin(dt * fs[FP_FINC], fs[FP_DTMAX]);
                alpha *= fs[FP_FALPHA];
            }
            fs[FS_BRANCH] = 1.0;
        } else {
            fs[FS_NPOS] = 0.0;
            fs[FS_NNEG] += 1.0;
            // too many P <= 0 steps in a row: with FP32 pair forces (a
            // switch threshold is set) that means their rounding floor has
            // been reached, so the FP64 phase takes over; otherwise FIRE fails
            if (fs[FS_NNEG] > fs[FP_NNEGMAX])
                status = fs[FP_SWITCH] > 0.0 ? FIRE_SWITCH : FIRE_NEGFAIL;
            // the back-off of dt stops short of dt_min (dt is left as it is
            // when f_dec dt would fall below it)
            if (!(fs[FP_INITDELAY] != 0.0 && fs[FS_ITER] < fs[FP_NDELAY])) {
                if (dt * fs[FP_FDEC] >= fs[FP_DTMIN]) dt *= fs[FP_FDEC];
                alpha = fs[FP_ALPHA0];
            }
            fs[FS_BRANCH] = 0.0;
        }
        // |v'| of v' = v + dt F/m (v = 0 after a P <= 0 step), expanded over
        // the sums of this reduction, for the mixing of every MD step
        const double vv = P > 0.0 ? red[R_VV] + 2.0 * dt * red[R_VF] + dt * dt * red[R_FF]
                                  : dt * dt * red[R_FF];
        fs[FS_VNORM] = sqrt(fmax(vv, 0.0));
        fs[FS_FNORM] = sqrt(red[R_FN]);
        fs[FS_DT] = dt;
        fs[FS_ALPHA] = alpha;
        if (status == FIRE_RUNNING) {
            fs[FS_ITER] += 1.0;
            fs[FS_PHASE_ITER] += 1.0;
        }
    }
    fs[FS_STATUS] = (double)status;
    return status;
}

}  // namespace hdmd
