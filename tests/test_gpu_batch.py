"""Batched path (many independent systems per call) vs the oracle and vs the
single-system path.  Tolerances as in test_gpu_parity: FP64 1e-6, FP32C 1e-4."""
import math

import numpy as np
import pytest

from oracle import OraclePPPM, estimate_g_ewald
from paper_1702_04250_gb300.workloads import batch_systems

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t

    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1702_04250_gb300 import build

    build.build()
    return t


def rel_rms(a, b):
    d = float(np.sum(b ** 2))
    return math.sqrt(float(np.sum((a - b) ** 2)) / d) if d > 0 else math.sqrt(float(np.sum(a ** 2)))


def small_batch():
    """Uneven sizes and orders; two systems share a mesh; one is empty and one
    has a single charge; non-cubic boxes and a ragged mesh."""
    r = np.random.default_rng(77)
    specs = [
        ((12.0, 12.0, 12.0), 600, 5, (16, 16, 16)),
        ((10.0, 11.0, 13.0), 350, 3, (12, 14, 18)),
        ((12.0, 12.0, 12.0), 900, 7, (16, 16, 16)),
        ((8.0, 8.0, 8.0), 0, 5, (8, 8, 8)),
        ((9.0, 9.0, 9.0), 1, 4, (10, 10, 10)),
        ((15.0, 14.0, 13.0), 1200, 5, (20, 17, 12)),
    ]
    out = []
    for box, n, P, mesh in specs:
        x = r.uniform(-2.0, max(box) + 2.0, (n, 3))
        q = r.normal(size=n) if n != 1 else np.array([1.0])
        out.append(dict(box=box, n=n, order=P, mesh=mesh, g_ewald=0.5, x=x, q=q))
    return out


def run_batch(torch, systems, mode, prec, graph=False, C=1.0, variant=None):
    from paper_1702_04250_gb300 import pppm

    dt = torch.float64 if prec == "fp64" else torch.float32
    b = pppm.PPPMBatch(systems, mode=mode, precision=prec, qqrd2e=C, graph=graph)
    if variant is not None:
        b.set_variant(variant)
    x = torch.tensor(np.concatenate([s["x"] for s in systems]).reshape(-1, 3), dtype=dt, device="cuda")
    q = torch.tensor(np.concatenate([s["q"] for s in systems]), dtype=dt, device="cuda")
    for _ in range(2 if graph else 1):
        f, ev = b.compute(x, q)
    b.sync()
    return b, f.double().cpu().numpy(), ev.cpu().numpy().copy()


@pytest.mark.parametrize("mode", ["ik", "ad"])
@pytest.mark.parametrize("prec", ["fp64", "fp32c"])
def test_small_batch_vs_oracle(torch, mode, prec):
    systems = small_batch()
    b, f, ev = run_batch(torch, systems, mode, prec)
    assert b.info()["mesh_classes"] == 5
    check_vs_oracle(b, f, ev, systems, mode, prec)


@pytest.mark.parametrize("mode", ["ik", "ad"])
@pytest.mark.parametrize("prec", ["fp64", "fp32c", "fp32"])
@pytest.mark.parametrize("variant", [0xFC0000, 0])
def test_small_batch_make_rho_layouts_vs_oracle(torch, mode, prec, variant):
    """make_rho over z-pairs of tiles for every order (bits 16 + P, the
    default) and one tile a CTA (mask 0): the batch's meshes have 1, 2 and 3
    z tiles, uniform and ragged (12 / 18 / 10 / 8 / 16 / 12 points along z)."""
    systems = small_batch()
    b, f, ev = run_batch(torch, systems, mode, prec, variant=variant)
    assert b.variant() == variant
    check_vs_oracle(b, f, ev, systems, mode, prec)


def check_vs_oracle(b, f, ev, systems, mode, prec):
    tol = 1e-6 if prec == "fp64" else 1e-4
    for s, sysd in enumerate(systems):
        lo, hi = b.offsets[s], b.offsets[s + 1]
        x, q = sysd["x"], sysd["q"]
        if prec != "fp64":
            x = x.astype(np.float32).astype(np.float64)
            q = q.astype(np.float32).astype(np.float64)
        ref = OraclePPPM(sysd["box"], sysd["mesh"], sysd["order"], sysd["g_ewald"], mode, 1.0).compute(x, q)
        if sysd["n"] == 0:
            assert np.all(ev[s] == 0.0)
            continue
        scale = max(np.abs(ref["f"]).max(), 1e-3)
        if sysd["n"] == 1:  # a lone charge: compare absolutely (ik force is ~0)
            assert np.abs(f[lo:hi] - ref["f"]).max() <= 10 * tol * scale
        else:
            assert rel_rms(f[lo:hi], ref["f"]) <= tol, (s, rel_rms(f[lo:hi], ref["f"]))
        assert abs(ev[s, 0] - ref["energy"]) <= tol * abs(ref["energy"]), s
        assert np.linalg.norm(ev[s, 1:] - ref["virial"]) <= tol * np.linalg.norm(ref["virial"]) + 1e-12, s


def test_batch_variants_and_autotune(torch):
    """Every order's make_rho brick (one or four copies, or one over z-pairs
    of tiles) and fieldforce (per particle through L1, or tile-staged from
    the planar field) give the same result; autotune returns a valid mask;
    FP64 batches refuse the brick-copy bits but take the fieldforce and
    tile-pair ones."""
    from paper_1702_04250_gb300 import pppm

    systems = small_batch()
    x = torch.tensor(np.concatenate([s["x"] for s in systems]).reshape(-1, 3), dtype=torch.float32, device="cuda")
    q = torch.tensor(np.concatenate([s["q"] for s in systems]), dtype=torch.float32, device="cuda")
    b = pppm.PPPMBatch(systems, mode="ik", precision="fp32c")
    outs = []
    for v in (0, 0xFC, 0xFC00, 0xFCFC, 0x0800 | 0x20, 0xFC0000, 0xFCFC00, 0x80 | 0x200000 | 0x0800):
        b.set_variant(v)
        f, ev = b.compute(x, q)
        b.sync()
        outs.append((f.double().cpu().numpy(), ev.cpu().numpy().copy()))
    for o in outs[1:]:
        assert rel_rms(o[0], outs[0][0]) < 1e-5
    choice = b.autotune(x, q)
    assert choice & ~0xFCFCFC == 0 and choice & (choice >> 16) & 0xFC == 0
    f, ev = b.compute(x, q)
    b.sync()
    assert rel_rms(f.double().cpu().numpy(), outs[0][0]) < 1e-5
    with pytest.raises(pppm.PPPMError):
        b.set_variant(1)
    for bad in (1 << 16, 1 << 24, 0x80 | 0x800000, 0x04 | 0x040000):  # unknown bits; pairs with copies
        with pytest.raises(pppm.PPPMError):
            b.set_variant(bad)
    b64 = pppm.PPPMBatch(systems, mode="ik", precision="fp64")
    with pytest.raises(pppm.PPPMError):
        b64.set_variant(1 << 5)
    x64, q64 = x.double(), q.double()
    f0, _ = b64.compute(x64, q64)
    b64.sync()
    f0 = f0.cpu().numpy()
    b64.set_variant(0xFC00)  # tile-staged fieldforce of every order, FP64
    f1, _ = b64.compute(x64, q64)
    b64.sync()
    assert rel_rms(f1.cpu().numpy(), f0) < 1e-12
    b64.set_variant(0xFC0000)  # tile pairs of every order, FP64
    f2, _ = b64.compute(x64, q64)
    b64.sync()
    assert rel_rms(f2.cpu().numpy(), f0) < 1e-12
    for mode in ("ad",):
        ba = pppm.PPPMBatch(systems, mode=mode, precision="fp32c")
        fa0, _ = ba.compute(x, q)
        ba.sync()
        fa0 = fa0.double().cpu().numpy()
        ba.set_variant(0xFC00)
        fa1, _ = ba.compute(x, q)
        ba.sync()
        assert rel_rms(fa1.double().cpu().numpy(), fa0) < 1e-5


def test_small_batch_graph_matches(torch):
    systems = small_batch()
    _, f0, ev0 = run_batch(torch, systems, "ik", "fp32c")
    _, f1, ev1 = run_batch(torch, systems, "ik", "fp32c", graph=True)
    # FP32C: the cross-tile flush adds floats in a run-dependent order
    assert rel_rms(f1, f0) < 1e-5
    for s in range(len(systems)):
        assert abs(ev1[s, 0] - ev0[s, 0]) <= 1e-6 * abs(ev0[s, 0]) + 1e-12
        assert np.linalg.norm(ev1[s, 1:] - ev0[s, 1:]) <= 1e-5 * np.linalg.norm(ev0[s, 1:]) + 1e-12


def c4_systems():
    ws = batch_systems()
    out = []
    for w in ws:
        g = estimate_g_ewald(w.rel_acc, w.r_cut, w.n, float(np.sum(w.q ** 2)), w.box)
        out.append(dict(box=w.box, n=w.n, order=w.order, mesh=w.mesh, g_ewald=g, x=w.x, q=w.q))
    return out


def test_c4_batch_vs_single_and_oracle(torch):
    """256 systems (N 500-20,000, meshes 16^3-64^3, orders 3/5/7), FP32C ik,
    one graph: every system vs its own single-system plan, every 32nd vs the
    FP64 oracle."""
    from paper_1702_04250_gb300 import pppm

    C = 332.06371
    systems = c4_systems()
    b, f, ev = run_batch(torch, systems, "ik", "fp32c", graph=True, C=C)
    worst = 0.0
    for s, sysd in enumerate(systems):
        lo, hi = b.offsets[s], b.offsets[s + 1]
        p = pppm.PPPM(sysd["box"], sysd["n"], sysd["order"], sysd["mesh"], sysd["g_ewald"], "ik", "fp32c", C)
        fs, evs = p.compute(torch.tensor(sysd["x"], dtype=torch.float32, device="cuda"),
                            torch.tensor(sysd["q"], dtype=torch.float32, device="cuda"))
        p.sync()
        e = rel_rms(f[lo:hi], fs.double().cpu().numpy())
        worst = max(worst, e)
        assert e < 1e-5, (s, e)
        # the energy is the mesh sum minus the self term C g/sqrt(pi) sum q^2,
        # which cancel to a few percent: the rounding scale is the mesh sum
        e_scale = abs(evs[0].item()) + C * sysd["g_ewald"] / math.sqrt(math.pi) * float(np.sum(sysd["q"] ** 2))
        assert abs(ev[s, 0] - evs[0].item()) < 1e-6 * e_scale, (s, ev[s, 0], evs[0].item(), e_scale)
        p.close()
        if s % 32 == 0:
            x = sysd["x"].astype(np.float32).astype(np.float64)
            q = sysd["q"].astype(np.float32).astype(np.float64)
            ref = OraclePPPM(sysd["box"], sysd["mesh"], sysd["order"], sysd["g_ewald"], "ik", C).compute(x, q)
            assert rel_rms(f[lo:hi], ref["f"]) < 1e-4, s
            assert abs(ev[s, 0] - ref["energy"]) < 1e-4 * e_scale, s
    print("c4 batch vs single-system plans: worst force rel RMS", worst)
