// Stopping and precision-switch rules of the ChebFD restart loop (host).
// The paper gives none; the readings implemented here:
//   - an in-window Ritz pair is converged when its residual <= tol;
//   - stop when the converged count reaches n_t (n_t > 0), or when it is
//     >= 1 and unchanged over three iterations while the smallest residual
//     of the unconverged in-window pairs did not halve in either of the last
//     two (nothing is still converging: the rest are spurious Ritz values);
//   - mixed policy: leave the fp32 filter when the count at switch_tol
//     reaches n_t, or stops growing while the smallest residual above
//     switch_tol did not halve (fp32 has stalled); the fp64 phase also stops
//     once at least that many pairs reach tol while the others still do not
//     improve (one fp64 sweep confirms what the fp32 phase found).
#pragma once

#include <vector>

namespace cfd {

constexpr double kNoPair = 1e300;   // "no unconverged in-window pair" (never improves)

struct ConvergenceTracker {
    int n_t = 0;
    bool mixed = false;
    bool low = false;                 // filter still in fp32
    int low_count = 0;                // in-window pairs at switch_tol when leaving fp32
    double mr_switch = kNoPair;       // smallest residual above switch_tol then
    std::vector<int> cnt, cnt_low;
    std::vector<double> mr, mr_low;

    void start(int target, bool mixed_policy) {
        n_t = target;
        mixed = mixed_policy;
        low = mixed_policy;
    }

    // One iteration's counts: cnt (residual <= tol) and cl (<= switch_tol)
    // of in-window pairs, m and ml the smallest residual above tol and above
    // switch_tol (kNoPair if none).  Returns true when converged.  While the
    // filter is still fp32 this only decides the switch (ready_to_switch()).
    bool update(int c, int cl, double m, double ml) {
        if (low) {
            cnt_low.push_back(cl);
            mr_low.push_back(ml);
            size_t h = cnt_low.size();
            bool stalled = h >= 2 && cl >= 1 && cnt_low[h - 1] <= cnt_low[h - 2] && mr_low[h - 1] > 0.5 * mr_low[h - 2];
            if ((n_t > 0 && cl >= n_t) || stalled) {
                switch_ready = true;
                low_count = cl;
                mr_switch = ml;
            }
            return false;
        }
        cnt.push_back(c);
        mr.push_back(m);
        size_t h = cnt.size();
        bool stable = h >= 3 && c >= 1 && cnt[h - 1] == cnt[h - 2] && cnt[h - 2] == cnt[h - 3] &&
                      mr[h - 1] > 0.5 * mr[h - 2] && mr[h - 2] > 0.5 * mr[h - 3];
        bool confirmed = mixed && low_count >= 1 && c >= low_count && m > 0.5 * mr_switch;
        return (n_t > 0 && c >= n_t) || stable || confirmed;
    }

    bool switch_ready = false;
    void leave_low() { low = false; }
};

}  // namespace cfd
