"""Host logic of the balanced gridding kernel's plan (no GPU): the order in which a warp's
(element, weight) entries are laid out.  Every lane must get exactly its own entries (the
sum of a cell does not depend on their order beyond FP32 rounding), padding entries must
carry a zero weight and a valid element, and the order must cut the shared-memory bank
conflicts of the gather, where the 8 lanes of a quarter-warp that read different elements
in the same 16-byte bank quad (element mod 8) are served one after another."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2609_03027_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.isfile(os.path.join(d, "include", "vector_types.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("host C++ compiler or CUDA headers not available")
    exe = str(tmp_path_factory.mktemp("host") / "order_entries")
    r = subprocess.run([cxx, "-O1", "-std=c++17", "-I", inc, "-I", CSRC,
                        os.path.join(ROOT, "tests", "host_order_entries.cpp"), os.path.join(CSRC, "plan.cpp"),
                        "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


def _run(exe, groups):
    lines = [str(len(groups))]
    for lists in groups:
        nmax = max(len(x) for x in lists)
        lines.append(f"{len(lists)} {nmax}")
        lines += [" ".join(map(str, [len(x)] + list(x))) for x in lists]
    r = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    out = []
    for lists, line in zip(groups, r.stdout.strip().split("\n")):
        nmax = max(len(x) for x in lists)
        v = np.array(line.split(), dtype=np.int64).reshape(nmax, 32, 2)  # [step][lane](element, payload)
        out.append(v)
    return out


def _quarter_wavefronts(elements):
    """[steps][32] elements -> sum over steps and quarter-warps of the 16-byte accesses
    that one bank quad must serve (distinct elements with the same element mod 8)."""
    t = 0
    for row in elements:
        for q0 in range(0, 32, 8):
            quads = {}
            for e in set(int(x) for x in row[q0:q0 + 8]):
                quads[e % 8] = quads.get(e % 8, 0) + 1
            t += max(quads.values())
    return t


def _element_order(lists):
    nmax = max(len(x) for x in lists)
    rows = np.zeros((nmax, 32), dtype=np.int64)
    for l, x in enumerate(lists):
        rows[:len(x), l] = x
    return rows


def _check_valid(lists, v, n_el):
    nmax = max(len(x) for x in lists)
    assert v.shape == (nmax, 32, 2)
    assert np.all((v[..., 0] >= 0) & (v[..., 0] < n_el))
    for l in range(32):
        col = v[:, l, :]
        real = col[col[:, 1] > 0]
        if l >= len(lists):
            assert len(real) == 0
            continue
        x = lists[l]
        # each input entry exactly once, with its own element
        assert sorted(real[:, 1].tolist()) == list(range(1, len(x) + 1)), l
        for e, pl in real:
            assert e == x[pl - 1]


def test_random_groups_keep_every_entry_and_pad_with_zero_weights(driver):
    rng = np.random.default_rng(7)
    groups = []
    for _ in range(60):
        members = int(rng.integers(1, 33))
        nmax = int(rng.integers(1, 14))
        lists = []
        for l in range(members):
            n = nmax if l == 0 else int(rng.integers(0, nmax + 1))
            lists.append(rng.choice(256, size=n, replace=False).tolist())
        groups.append(lists)
    for lists, v in zip(groups, _run(driver, groups)):
        _check_valid(lists, v, 256)


def test_footprint_lists_order_cuts_bank_conflicts(driver):
    # cells of a K x K footprint gridding of a random disc layout, grouped by list length as
    # the plan does: neighbouring cells share elements, so broadcasts and distinct quads exist
    rng = np.random.default_rng(3)
    A, K, side = 256, 5, 48
    pos = rng.uniform(0, side - K, size=(A, 2))
    first = np.floor(pos).astype(int)
    cells = {}
    for e in range(A):
        for ty in range(K):
            for tx in range(K):
                cells.setdefault((first[e, 1] + ty, first[e, 0] + tx), []).append(e)
    keys = sorted(cells, key=lambda c: (-len(cells[c]), c))
    groups = [[cells[c] for c in keys[i:i + 32]] for i in range(0, len(keys), 32)]
    outs = _run(driver, groups)
    ordered = plain = 0
    for lists, v in zip(groups, outs):
        _check_valid(lists, v, A)
        ordered += _quarter_wavefronts(v[..., 0])
        plain += _quarter_wavefronts(_element_order(lists))
    assert ordered <= 0.85 * plain, (ordered, plain)


def test_single_lane_and_single_entry_groups(driver):
    groups = [[[5]], [[3, 11, 19]], [[0], [8], [16], [24]]]
    outs = _run(driver, groups)
    for lists, v in zip(groups, outs):
        _check_valid(lists, v, 32)
    # one entry per lane on the same quad: nothing to reorder, every lane keeps its element
    assert outs[2][0, :4, 0].tolist() == [0, 8, 16, 24]
