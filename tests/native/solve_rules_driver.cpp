// Host driver for the restart loop's stopping and precision-switch rules
// (csrc/solve_rules.h), used by tests/test_solve_rules.py on the CPU.
// Usage: solve_rules_driver MIXED N_T  [c cl m ml]...  (one quadruple per
// iteration: in-window counts at tol and at switch_tol, smallest residuals
// above them).  Prints "iteration low done" per iteration, the way the
// solve loop consults the tracker, and stops at the first "done".
#include <cstdio>
#include <cstdlib>

#include "solve_rules.h"

int main(int argc, char **argv) {
    if (argc < 3) return 2;
    cfd::ConvergenceTracker tr;
    tr.start(std::atoi(argv[2]), std::atoi(argv[1]) != 0);
    for (int i = 3, it = 1; i + 3 < argc; i += 4, ++it) {
        const bool low = tr.low;
        const bool done = tr.update(std::atoi(argv[i]), std::atoi(argv[i + 1]), std::atof(argv[i + 2]),
                                    std::atof(argv[i + 3]));
        std::printf("%d %d %d\n", it, low ? 1 : 0, done ? 1 : 0);
        if (done) return 0;
        if (tr.low && tr.switch_ready) tr.leave_low();
    }
    return 0;
}
