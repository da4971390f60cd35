"""The rule that ends the mixed phase of kgs_solve and kgs_batch_solve
(kgs::SolveSwitch in csrc/kgs_switch.h), exercised on the host: the header
is compiled into a small driver with the host C++ compiler and fed
synthetic chunk-end residual sequences.

What the rule must do: stop at a flat noise floor after a fixed number of
chunks that depends on where the floor lies (two below 3e-6, six up to 1e-3,
twenty above), never stop while the residual keeps falling by more than 10%
a chunk, and not take the bumps of a small-Kn residual -- a damped
oscillation of the iteration with a period of about 25 iterations, five
chunks -- for a floor: between 3e-6 and 1e-3 the six-chunk patience spans a
whole period, so such a descent is followed down into the floor band.
"""
import math
import os
import shutil
import subprocess

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1810_00348_gb300", "csrc")

DRIVER = r"""
#include <cstdio>
#include <iostream>
#include <sstream>
#include <string>
#include "kgs_switch.h"
int main()
{
    std::string line;
    while (std::getline(std::cin, line)) {
        std::istringstream in(line);
        kgs::SolveSwitch sw;
        double r;
        int chunk = 0, stop = 0;
        while (in >> r) {
            ++chunk;
            if (sw.stalled_after(r)) { stop = chunk; break; }
        }
        std::printf("%d\n", stop);
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def switch(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("switch")
    src, exe = d / "driver.cpp", d / "driver"
    src.write_text(DRIVER)
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def run(seqs):
        text = "\n".join(" ".join("%.17g" % r for r in s) for s in seqs) + "\n"
        out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True).stdout
        return [int(v) for v in out.split()]

    return run


def jitter(level, n):
    # a flat floor with fluctuations of +-4%: never a 10% improvement
    return [level * (1.0 + 0.04 * math.sin(1.3 * c)) for c in range(n)]


@pytest.mark.parametrize("level,stop", [(1e-6, 3), (2.5e-6, 3), (4e-6, 7), (1e-5, 7), (9e-4, 7), (1.1e-3, 21),
                                        (1e-2, 21)])
def test_flat_floor_stops_after_the_band_patience(switch, level, stop):
    # the first chunk sets the best value; then 2, 6 or 20 chunks without progress
    assert switch([jitter(level, 40)]) == [stop]


def test_steady_descent_never_stops(switch):
    seqs = [[0.8 ** c for c in range(80)],            # 0.8 a chunk: from 1 to 1e-8
            [1e-3 * 0.89 ** c for c in range(120)]]   # just over 10% a chunk
    assert switch(seqs) == [0, 0]


def test_progress_resets_the_count(switch):
    # in the middle band: five stalled chunks, one chunk of progress, five more
    s = [1e-4] + [1e-4] * 5 + [0.85e-4] + [0.85e-4] * 5 + [0.85e-4]
    assert switch([s]) == [13]


def small_kn_descent(phase, tau, amp, floor=1e-6, chunks=90):
    # chunk-end residuals (every 5th iteration) of a damped oscillation with a
    # period of 25 iterations on a falling trend, over a noise floor
    out = []
    for c in range(1, chunks + 1):
        k = 5 * c
        trend = 1e-2 * math.exp(-k / tau) * (1.0 + amp * math.sin(2.0 * math.pi * k / 25.0 + phase))
        out.append(trend + floor * (1.0 + 0.05 * math.sin(1.7 * c)))
    return out


@pytest.mark.parametrize("tau", [18.0, 22.0, 30.0, 45.0])
def test_small_kn_bumps_are_not_taken_for_the_floor(switch, tau):
    seqs = [small_kn_descent(phase, tau, amp) for phase in (0.0, 1.0, 2.0, 3.0, 4.0, 5.0) for amp in (0.5, 0.85)]
    stops = switch(seqs)
    for s, stop in zip(seqs, stops):
        assert stop > 0
        # the phase ends in the floor band, not at a bump above it
        assert s[stop - 1] < 3e-6, (tau, stop, s[stop - 1])
