"""The oracle's context windows (oracle_contexts) pinned to things other than
itself: worked examples derived by hand from the definition, an independent
construction from numpy sliding windows, the closed-form number of SkipGram
pairs of a row, and the symmetry of the pairs; a planted off-by-one in a copy
of the source fails them."""
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "contexts_examples.txt")
SRC = os.path.join(os.path.dirname(oracle.__file__), "walk_oracle.c")


def golden_cases():
    cases, cur = [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        if key == "window":
            cur = {"window": int(vals[0]), "ctx": []}
        elif key == "row":
            cur["row"] = [int(v) for v in vals]
        elif key == "ctx":
            cur["ctx"].append([int(v) for v in vals])
        elif key == "end":
            cases.append(cur)
    return cases


def sliding_construction(rows, w):
    """Pad each row with w entries of -1 on both sides, take every window of
    2w + 1 consecutive entries, drop its middle: the context of the middle."""
    n, L = rows.shape
    pad = np.full((n, L + 2 * w), -1, np.int32)
    pad[:, w:w + L] = rows
    win = np.lib.stride_tricks.sliding_window_view(pad, 2 * w + 1, axis=1)   # [n, L, 2w+1]
    ctx = np.concatenate([win[:, :, :w], win[:, :, w + 1:]], axis=2).copy()
    ctx[rows < 0] = -1
    return ctx


def random_rows(rng, n, L, nodes=50):
    rows = rng.integers(0, nodes, (n, L)).astype(np.int32)
    for r in range(n):                       # -1 suffixes: dead ends at random points
        cut = int(rng.integers(0, L + 1)) if rng.random() < 0.4 else L
        rows[r, cut:] = -1
    return rows


def pin_battery(lib):
    failed = []
    for c in golden_cases():
        got = oracle.contexts(np.array([c["row"]], np.int32), c["window"], lib=lib)[0]
        if not np.array_equal(got, np.array(c["ctx"], np.int32)):
            failed.append("golden")
            break
    rng = np.random.default_rng(3)
    for w in (1, 2, 5, 9):
        for L in (1, 3, 10, 40):
            rows = random_rows(rng, 30, L)
            got = oracle.contexts(rows, w, lib=lib)
            if not np.array_equal(got, sliding_construction(rows, w)):
                failed.append(f"sliding(w={w},L={L})")
            # closed form: a row with n valid nodes has sum_i min(i, w) + min(n-1-i, w) pairs
            nvalid = (rows >= 0).sum(axis=1)
            want = [sum(min(i, w) + min(n - 1 - i, w) for i in range(n)) for n in nvalid]
            if not np.array_equal((got >= 0).sum(axis=(1, 2)), np.array(want)):
                failed.append(f"count(w={w},L={L})")
            # symmetry: entry j < w of centre i is position a = i - w + j, and then
            # entry w + (i - a) - 1 of centre a is the centre i
            for r in range(len(rows)):
                for i in range(L):
                    for j in range(w):
                        a = i - w + j
                        if got[r, i, j] >= 0 and got[r, a, w + (i - a) - 1] != rows[r, i]:
                            failed.append(f"symmetry(w={w},L={L})")
                            break
    return sorted(set(failed))


def test_oracle_contexts_pass_their_pins():
    assert pin_battery(oracle.load()) == []


PLANTS = {
    "window_off_by_one": ("(int64_t)i - window + j", "(int64_t)i - window + j + 1"),
    "after_side_from_centre": ("(int64_t)i + 1 + (j - window)", "(int64_t)i + (j - window)"),
    "dead_centre_kept": ("if (row[i] >= 0 && pos >= 0", "if (pos >= 0"),
}


@pytest.mark.parametrize("name", sorted(PLANTS))
def test_planted_context_mistake_is_caught(name, tmp_path):
    old, new = PLANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    mutated = tmp_path / "walk_oracle_planted.c"
    mutated.write_text(src.replace(old, new))
    so = oracle.compile_oracle(str(mutated), str(tmp_path / "liboracle_planted.so"))
    assert pin_battery(oracle.load(so)), f"planted mistake {name} escaped every pin"
