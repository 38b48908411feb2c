"""Host logic of the autotuner and of the binding's constants (no GPU):

* every ABC_* constant the binding defines has the value the C header gives it;
* the autotuner offers each knob only where the library applies it (the node-major
  chain only on the tensor-core path of an order-1 limit-fit step with a multiple of 32
  orbitals, the Gamma copy only for complex64 at radius 1 with even rows, ...), every
  candidate of a group sets the same knobs (so that the group's winner leaves no knob of
  a loser behind), and the first candidate of the forward group is the library default;
* describe() names every knob the groups use."""
import os
import re

import pytest

from paper_1908_02456_gb300 import abc, tune

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "abc.h")


def header_defines():
    out = {}
    for line in open(HEADER):
        m = re.match(r"#define (ABC_\w+) (-?\d+)", line)
        if m:
            out[m.group(1)] = int(m.group(2))
    return out


def test_binding_constants_match_header():
    d = header_defines()
    pairs = {"ABC_TUNE_" + n[5:]: getattr(abc, n) for n in dir(abc) if n.startswith("TUNE_")}
    pairs.update({"ABC_KERNEL_" + n[7:]: getattr(abc, n) for n in dir(abc) if n.startswith("KERNEL_")})
    pairs.update({"ABC_FIT1_" + n[5:]: getattr(abc, n) for n in dir(abc) if n.startswith("FIT1_")})
    assert len(pairs) >= 20
    for name, value in pairs.items():
        assert name in d, name
        assert d[name] == value, name


class FakeCtx:
    """The attributes knob_groups reads from an abc.Context."""

    def __init__(self, precision, order=1, fit1=abc.FIT1_LIMIT, shape=(96, 96, 96), radius=1, tiles=0):
        self.precision, self.order, self.fit1, self.shape, self.radius = precision, order, fit1, shape, radius
        self.tiles = tiles

    def get_tuning(self, key):
        assert key == abc.TUNE_TILE_COUNT
        return self.tiles


def knobs_of(groups):
    return [set().union(*(c.keys() for c in g)) for g in groups]


def all_candidates(groups):
    return [c for g in groups for c in g]


@pytest.mark.parametrize("b", [128, 64, 32])
def test_node_major_chain_offered_on_the_tensor_core_path(b):
    groups = tune.knob_groups(FakeCtx(abc.C64_SPLIT_FP16), b)
    fwd = [g for g in groups if any(abc.TUNE_LANES in c for c in g)]
    assert len(fwd) == 1
    lanes = sorted({c[abc.TUNE_LANES] for c in fwd[0]})
    assert lanes == [0, 1, 2, 3, 4, 5]
    assert fwd[0][0] == {abc.TUNE_FORWARD_RW: 0, abc.TUNE_GAMMA_COPY: 0, abc.TUNE_LANES: 0}
    # the node-major forms are offered with and without the Gamma copy
    assert {(c[abc.TUNE_LANES], c[abc.TUNE_GAMMA_COPY]) for c in fwd[0] if c[abc.TUNE_LANES]} == \
        {(ln, gc) for ln in range(1, 6) for gc in (0, 1)}


@pytest.mark.parametrize("ctx,b", [(FakeCtx(abc.C64_SPLIT_FP16), 40),          # not a multiple of 32
                                   (FakeCtx(abc.C64_SPLIT_FP16), 8),
                                   (FakeCtx(abc.C64_FP32), 128),               # no tensor cores
                                   (FakeCtx(abc.FP64), 128),
                                   (FakeCtx(abc.C64_SPLIT_FP16, fit1=abc.FIT1_TWO_POINT), 128),
                                   (FakeCtx(abc.C64_SPLIT_FP16, order=0), 128),
                                   (FakeCtx(abc.C64_SPLIT_FP16, order=2), 128)])
def test_node_major_chain_not_offered_elsewhere(ctx, b):
    assert all(abc.TUNE_LANES not in c for c in all_candidates(tune.knob_groups(ctx, b)))


def test_groups_set_the_same_knobs_in_every_candidate():
    for ctx, b in [(FakeCtx(abc.C64_SPLIT_FP16), 128), (FakeCtx(abc.C64_3XTF32, shape=(64, 64, 64)), 32),
                   (FakeCtx(abc.C64_FP32, shape=(64, 64, 64)), 1), (FakeCtx(abc.C64_FP32, tiles=1586), 1),
                   (FakeCtx(abc.C64_FP32, shape=(31, 31, 31), radius=3), 4),
                   (FakeCtx(abc.FP64, shape=(16, 16, 16)), 4)]:
        for g in tune.knob_groups(ctx, b):
            keys = [set(c) for c in g]
            assert len(g) >= 2, g
            assert all(k == keys[0] for k in keys), g
            assert len({tuple(sorted(c.items())) for c in g}) == len(g), g     # no duplicates


def test_gamma_copy_needs_complex64_radius1_even_rows():
    for ctx in (FakeCtx(abc.FP64), FakeCtx(abc.C64_FP32, radius=3), FakeCtx(abc.C64_FP32, shape=(31, 31, 31))):
        assert all(c.get(abc.TUNE_GAMMA_COPY, 0) == 0 for c in all_candidates(tune.knob_groups(ctx, 8)))
    assert any(c.get(abc.TUNE_GAMMA_COPY) == 1 for c in all_candidates(tune.knob_groups(FakeCtx(abc.C64_FP32), 8)))


def test_gemm_group_only_on_tensor_core_forms():
    for prec in (abc.C64_3XTF32, abc.C64_SPLIT_FP16):
        gk = knobs_of(tune.knob_groups(FakeCtx(prec), 32))
        assert {abc.TUNE_GEMM_TILE, abc.TUNE_GEMM_SPLIT} in gk
    for ctx, b in [(FakeCtx(abc.C64_FP32), 32), (FakeCtx(abc.C64_SPLIT_FP16), 1), (FakeCtx(abc.FP64), 32)]:
        assert all(abc.TUNE_GEMM_TILE not in c for c in all_candidates(tune.knob_groups(ctx, b)))


def test_one_orbital_offers_the_early_start_only_with_tiles():
    with_tiles = all_candidates(tune.knob_groups(FakeCtx(abc.C64_FP32, tiles=1586), 1))
    without = all_candidates(tune.knob_groups(FakeCtx(abc.C64_FP32, tiles=0), 1))
    assert any(abc.TUNE_PDL in c for c in with_tiles)
    assert all(abc.TUNE_PDL not in c for c in without)


def test_describe_names_every_knob():
    used = set()
    for ctx, b in [(FakeCtx(abc.C64_SPLIT_FP16), 128), (FakeCtx(abc.C64_FP32, tiles=1586), 1)]:
        for c in all_candidates(tune.knob_groups(ctx, b)):
            used |= set(c)
    names = tune.describe({k: 0 for k in used})
    assert all(not n.isdigit() for n in names), names
