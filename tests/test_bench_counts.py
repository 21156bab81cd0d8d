"""The kernel launches bench.py claims for its timed steps (`gpu_launches`),
against the launch sequence of one step on each path: the step kernel; the
ghost fill after the tiled kernels' steps; on the in-place tiled path the
(phi, T) pass, and a ghost refresh and a fold around the steps from even
levels; the RK stages of the finite-difference energy solvers."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _by_step(kernel, thermal, steps, warmup):
    """Count launch by launch, one level at a time."""
    rk = {"RK2": 1, "RK4": 3}.get(thermal, 0)
    n = 0
    for level in range(warmup, warmup + steps):
        if kernel in ("skew", "bulk"):
            n += 1 + 1                      # step kernel, ghost fill
        elif kernel == "generic":
            n += 1
        elif kernel == "aa":
            n += 2                          # (phi, T) pass, in-place step
        elif kernel == "aa_tiled":
            n += 2 + (2 if level % 2 == 0 else 0)   # + ghost refresh and fold from even levels
        n += rk
    return n


def test_timed_launch_count_matches_the_step_sequence():
    b = _bench()
    for kernel in ("skew", "bulk", "generic", "aa", "aa_tiled"):
        for thermal in ("D3Q7", "D3Q27", "RK2", "RK4"):
            for steps in (1, 2, 5, 30):
                for warmup in (0, 3, 4, 5):
                    got = b.timed_launch_count(kernel, thermal, steps, warmup)
                    assert got == _by_step(kernel, thermal, steps, warmup), (kernel, thermal, steps, warmup, got)


def test_headline_launches_per_step():
    b = _bench()
    assert b.timed_launch_count("skew", "D3Q7", 30, 5) == 60
    assert b.timed_launch_count("skew", "RK4", 10, 3) == 50
