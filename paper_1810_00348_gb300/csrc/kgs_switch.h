// kgs_switch.h -- when a mixed-then-FP64 solve leaves the mixed phase
// (kgs_solve, kgs_batch_solve).  Plain C++ with no CUDA, so that the rule can
// be exercised on the host alone.  Not part of the public ABI.
//
// Mixed iterations run in chunks of SOLVE_CHUNK; after each chunk the
// residual r of its last iteration is passed to SolveSwitch::stalled_after.
// The mixed phase ends once r has not fallen below SOLVE_PROGRESS x its best
// value for solve_patience(r) chunks in a row:
//  * r >= SOLVE_NEAR_FLOOR: twenty chunks (small-Kn solves can first rise for
//    a while);
//  * SOLVE_FLOOR_BAND <= r < SOLVE_NEAR_FLOOR: six chunks.  At small Kn the
//    residual falls with bumps: a slowly damped oscillation of the iteration
//    whose period is about 25 iterations (Kn 0.05 cavity: the residual rises
//    from 3e-4 to 6e-4 and takes 20 iterations to fall back below its
//    previous best), which two chunks mistook for the noise floor;
//  * r < SOLVE_FLOOR_BAND: two chunks.  The mixed form's own floor (rounding
//    noise of the smallest field, about 1e-6 with the deviation-form source)
//    lies here, and there a stall is the floor.
#pragma once

#include <algorithm>

namespace kgs {

constexpr int SOLVE_CHUNK = 5;
constexpr double SOLVE_PROGRESS = 0.9;
constexpr double SOLVE_NEAR_FLOOR = 1e-3;
constexpr double SOLVE_FLOOR_BAND = 3e-6;
constexpr int SOLVE_PATIENCE_FAR = 20;
constexpr int SOLVE_PATIENCE_MID = 6;
constexpr int SOLVE_PATIENCE = 2;

inline int solve_patience(double r)
{
    if (r >= SOLVE_NEAR_FLOOR) return SOLVE_PATIENCE_FAR;
    return r >= SOLVE_FLOOR_BAND ? SOLVE_PATIENCE_MID : SOLVE_PATIENCE;
}

// The stall detector of one instance.
struct SolveSwitch {
    double best = 1e300;  // lowest chunk-end residual so far
    int stalled = 0;      // chunks in a row without progress
    // r: residual at the end of a chunk.  Returns true when the mixed phase
    // should end.
    bool stalled_after(double r)
    {
        bool stop = false;
        if (r < SOLVE_PROGRESS * best)
            stalled = 0;
        else
            stop = ++stalled >= solve_patience(r);
        best = std::min(best, r);
        return stop;
    }
};

}  // namespace kgs
