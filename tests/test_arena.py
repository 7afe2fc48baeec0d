"""The render server's device arena (first fit over offsets, neighbours
merged on release), host logic on the CPU: the C++ allocator of
`csrc/arena.h`, driven through `tests/arena_driver.cpp`, against a plain
Python model of first fit on a sorted list of free ranges."""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2311_17089_gb300", "csrc")


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("arena") / "arena_driver")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-I", CSRC,
                    os.path.join(HERE, "arena_driver.cpp"), "-o", exe], check=True)
    return exe


class Model:
    """First fit by lowest offset; a release merges with adjacent free
    ranges.  Free ranges as a sorted list of [offset, size]."""

    def __init__(self, size):
        self.size, self.used, self.peak = size, 0, 0
        self.free = [[0, size]] if size else []

    def alloc(self, b):
        for k, (o, s) in enumerate(self.free):
            if s >= b:
                if s == b:
                    del self.free[k]
                else:
                    self.free[k] = [o + b, s - b]
                self.used += b
                self.peak = max(self.peak, self.used)
                return o
        return None

    def release(self, o, b):
        self.used -= b
        self.free.append([o, b])
        self.free.sort()
        merged = []
        for r in self.free:
            if merged and merged[-1][0] + merged[-1][1] == r[0]:
                merged[-1][1] += r[1]
            else:
                merged.append(r)
        self.free = merged

    def state(self):
        return f"{self.size} {self.used} {self.peak}" + "".join(
            f" {o}:{s}" for o, s in self.free)


def run(driver, lines):
    out = subprocess.run([driver], input="\n".join(lines) + "\n", capture_output=True,
                         text=True, check=True).stdout.splitlines()
    assert len(out) == len(lines)
    return out


@pytest.mark.parametrize("seed", range(6))
def test_arena_matches_first_fit_model(driver, seed):
    rng = np.random.default_rng(seed)
    size = int(rng.choice([1 << 12, 1 << 20, 3 * (1 << 30)]))
    unit = max(size // 64, 1)
    m = Model(size)
    live, lines, expect = [], [f"init {size}"], ["ok"]
    for _ in range(1500):
        r = rng.random()
        if r < 0.55 or not live:
            b = int(rng.integers(1, 12)) * unit + int(rng.integers(0, 3)) * 256
            lines.append(f"alloc {b}")
            o = m.alloc(b)
            expect.append("fail" if o is None else f"ok {o}")
            if o is not None:
                live.append((o, b))
        elif r < 0.97:
            o, b = live.pop(int(rng.integers(0, len(live))))
            lines.append(f"release {o} {b}")
            m.release(o, b)
            expect.append("ok")
        else:
            lines.append("state")
            expect.append(m.state())
    while live:  # everything back: one free range, nothing used
        o, b = live.pop(int(rng.integers(0, len(live))))
        lines.append(f"release {o} {b}")
        m.release(o, b)
        expect.append("ok")
    lines.append("state")
    expect.append(m.state())
    assert run(driver, lines) == expect
    assert expect[-1].split()[1] == "0" and expect[-1].endswith(f" 0:{size}")


def test_arena_edges(driver):
    """Exact fit, a request larger than the arena, a zero-size arena, and
    merging from both sides into one range."""
    lines = ["init 1000", "alloc 1000", "alloc 1", "state", "release 0 1000", "state",
             "alloc 1001", "alloc 300", "alloc 300", "alloc 400", "release 0 300",
             "release 600 400", "state", "release 300 300", "state", "init 0", "alloc 1",
             "state"]
    assert run(driver, lines) == [
        "ok", "ok 0", "fail", "1000 1000 1000", "ok", "1000 0 1000 0:1000",
        "fail", "ok 0", "ok 300", "ok 600", "ok", "ok", "1000 300 1000 0:300 600:400",
        "ok", "1000 0 1000 0:1000", "ok", "fail", "0 0 0"]
