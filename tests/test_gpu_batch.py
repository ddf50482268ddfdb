"""Batched persistent launch (rbe2d_batch_*): every system's forces and energies equal
those of the single-system path with the same parameters, seed and step (up to float32
summation order), match the FP64 oracle within the FP32 bar (rel-L2 <= 1e-4), are bitwise
reproducible, and survive the autotuner's choice."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O
from paper_2405_06333_gb300 import binding as B
from paper_2405_06333_gb300.synthetic import batched_systems, positions_charges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_06333_gb300 import build
    build.build()
    yield


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def make_batch(n_sys, n_hi, P=200, seed=2):
    systems = batched_systems(n_sys=n_sys, seed=seed, n_hi=n_hi)
    params, pos, q, off = [], [], [], [0]
    for i, sy in enumerate(systems):
        p_, q_ = positions_charges(sy["N"], sy["Lx"], sy["Ly"], sy["H"], seed=sy["pos_seed"])
        alpha = (sy["N"] / (sy["Lx"] * sy["Ly"] * sy["H"])) ** (1 / 3)
        params.append(B.rbe2d_params(Lx=sy["Lx"], Ly=sy["Ly"], H=sy["H"], Lz=-1, gamma_top=sy["gamma_top"],
                                     gamma_bot=sy["gamma_bot"], M=-1, alpha=alpha, r_c=-1, P=P, seed=100 + i,
                                     eps=1e-4, precision=B.RBE2D_FP32_MIXED, coulomb_k=1.0, real_space=0))
        pos.append(p_); q.append(q_); off.append(off[-1] + sy["N"])
    return systems, params, np.concatenate(pos), np.concatenate(q), np.array(off, dtype=np.int64)


def single(p, pos, q, step):
    ctx = B.rbe2d_init(p, len(q), torch.cuda.current_stream())
    k = torch.empty((p.P, 3), dtype=torch.int32, device="cuda")
    B.rbe2d_sample_k(ctx, step, k)
    F = torch.empty((len(q), 3), dtype=torch.float32, device="cuda")
    e = torch.zeros(4, dtype=torch.float64, device="cuda")
    B.rbe2d_force(ctx, len(q), torch.as_tensor(pos, device="cuda"), torch.as_tensor(q, device="cuda"),
                  B.RBE2D_KSPACE | B.RBE2D_IBC | B.RBE2D_ENERGY, F, None, e)
    d = B.rbe2d_get_derived(ctx)
    torch.cuda.synchronize()
    B.rbe2d_destroy(ctx)
    return F.cpu().numpy(), e.cpu().numpy(), k.cpu().numpy(), d


def test_batch_equals_single_system_path_and_oracle():
    systems, params, pos, q, off = make_batch(10, 3000)
    b = B.rbe2d_batch_init(params, off)
    F = torch.empty((off[-1], 3), dtype=torch.float32, device="cuda")
    E = torch.zeros((len(systems), 4), dtype=torch.float64, device="cuda")
    P_, Q_ = torch.as_tensor(pos, device="cuda"), torch.as_tensor(q, device="cuda")
    step = 3
    B.rbe2d_batch_force(b, step, P_, Q_, B.RBE2D_KSPACE | B.RBE2D_IBC | B.RBE2D_ENERGY, F, E)
    B.rbe2d_batch_sync_status(b)
    Fb, Eb = F.cpu().numpy(), E.cpu().numpy()
    for s in range(len(systems)):
        sl = slice(off[s], off[s + 1])
        Fs, es, k, d = single(params[s], pos[sl], q[sl], step)
        assert rel_l2(Fb[sl], Fs) < 1e-5, s
        assert Eb[s, 0] == pytest.approx(es[0], rel=1e-6)
        # both paths sum mu = sum q z in float64 (in different orders)
        assert Eb[s, 2] == pytest.approx(es[2], rel=1e-9, abs=1e-12)
        if s < 3:
            sy = systems[s]
            osys = O.System(Lx=sy["Lx"], Ly=sy["Ly"], H=sy["H"], Lz=d["Lz"], gamma_top=sy["gamma_top"],
                            gamma_bot=sy["gamma_bot"], alpha=d["alpha"], M=d["M"])
            ref = O.rbe(osys, pos[sl], q[sl], k, mode=1)
            assert rel_l2(Fb[sl], ref["force"]) < 1e-4, s
    # bitwise reproducible
    F2 = torch.empty_like(F)
    B.rbe2d_batch_force(b, step, P_, Q_, B.RBE2D_KSPACE | B.RBE2D_IBC, F2)
    torch.cuda.synchronize()
    assert torch.equal(F, F2)
    # the autotuner keeps the results (the fold order does not depend on chunk sizes only
    # up to float32 rounding) and reports its choice
    choice = B.rbe2d_batch_autotune(b, P_, Q_, F2)
    assert choice["sf_chunk"] in (256, 512, 1024, 2048) and choice["f_chunk"] in (256, 512, 1024)
    assert choice["variant"] in (0, 1, 2, 3)
    B.rbe2d_batch_force(b, step, P_, Q_, B.RBE2D_KSPACE | B.RBE2D_IBC, F2)
    B.rbe2d_batch_sync_status(b)
    assert rel_l2(F2.cpu().numpy(), Fb) < 1e-5
    B.rbe2d_batch_destroy(b)


@pytest.mark.parametrize("Ps", [
    (1, 16, 17, 33, 100, 128),        # 1 wave vector slot per thread (P_max <= 128)
    (129, 136, 150, 200, 232, 256),   # 2 slots
    (260, 300, 340, 488, 500, 512),   # 4 slots
])
def test_every_last_group_width_matches_the_single_system_path(Ps):
    """Systems with their own batch sizes: the structure-factor items hold ceil(P / 32)
    groups of 32 wave vectors, and a last group of at most 16 (P = 1, 16, 33, 100, 136,
    200, 232, 260, 300, 488 here) runs on split lanes of warp 3; the others (17, 128, 150,
    256, 340, 500, 512) on ordinary slots.  Every system equals the single-system path,
    and the first matches the FP64 oracle."""
    systems = batched_systems(n_sys=len(Ps), seed=7, n_lo=400, n_hi=2400)
    params, pos, q, off = [], [], [], [0]
    for i, (sy, P) in enumerate(zip(systems, Ps)):
        p_, q_ = positions_charges(sy["N"], sy["Lx"], sy["Ly"], sy["H"], seed=sy["pos_seed"])
        alpha = (sy["N"] / (sy["Lx"] * sy["Ly"] * sy["H"])) ** (1 / 3)
        params.append(B.rbe2d_params(Lx=sy["Lx"], Ly=sy["Ly"], H=sy["H"], Lz=-1, gamma_top=sy["gamma_top"],
                                     gamma_bot=sy["gamma_bot"], M=-1, alpha=alpha, r_c=-1, P=P, seed=300 + i,
                                     eps=1e-4, precision=B.RBE2D_FP32_MIXED, coulomb_k=1.0, real_space=0))
        pos.append(p_); q.append(q_); off.append(off[-1] + sy["N"])
    pos, q, off = np.concatenate(pos), np.concatenate(q), np.array(off, dtype=np.int64)
    b = B.rbe2d_batch_init(params, off)
    F = torch.empty((off[-1], 3), dtype=torch.float32, device="cuda")
    P_, Q_ = torch.as_tensor(pos, device="cuda"), torch.as_tensor(q, device="cuda")
    step = 2
    # the register cap (variant bit 0) exists for P_max <= 256 only
    for variant in ((0, 1, 2, 3) if max(Ps) <= 256 else (0, 2)):
        B.rbe2d_batch_set_tuning(b, 256, 256, 152 * 2, variant)
        B.rbe2d_batch_force(b, step, P_, Q_, B.RBE2D_KSPACE | B.RBE2D_IBC, F)
        B.rbe2d_batch_sync_status(b)
        Fb = F.cpu().numpy()
        for s in range(len(Ps)):
            sl = slice(off[s], off[s + 1])
            Fs, _, k, d = single(params[s], pos[sl], q[sl], step)
            assert rel_l2(Fb[sl], Fs) < 1e-5, (variant, Ps[s])
            if s == 0 and variant == 2:
                sy = systems[s]
                osys = O.System(Lx=sy["Lx"], Ly=sy["Ly"], H=sy["H"], Lz=d["Lz"], gamma_top=sy["gamma_top"],
                                gamma_bot=sy["gamma_bot"], alpha=d["alpha"], M=d["M"])
                assert rel_l2(Fb[sl], O.rbe(osys, pos[sl], q[sl], k, mode=1)["force"]) < 1e-4
    B.rbe2d_batch_destroy(b)


def test_full_512_system_workload_spot_checks():
    systems, params, pos, q, off = make_batch(512, 20000)
    b = B.rbe2d_batch_init(params, off)
    F = torch.empty((off[-1], 3), dtype=torch.float32, device="cuda")
    P_, Q_ = torch.as_tensor(pos, device="cuda"), torch.as_tensor(q, device="cuda")
    B.rbe2d_batch_force(b, 0, P_, Q_, B.RBE2D_KSPACE | B.RBE2D_IBC, F)
    B.rbe2d_batch_sync_status(b)
    Fb = F.cpu().numpy()
    assert np.all(np.isfinite(Fb))
    for s in (0, 255, 511):
        sl = slice(off[s], off[s + 1])
        Fs, _, _, _ = single(params[s], pos[sl], q[sl], 0)
        assert rel_l2(Fb[sl], Fs) < 1e-5, s
    B.rbe2d_batch_destroy(b)


def test_a_withheld_system_times_out_and_the_others_are_evaluated():
    """Failure detection of the persistent launch: one system's fold is kept from
    publishing its ready flag (host-side injection), its force items give up after the
    1 ms bound and report RBE2D_ETIMEOUT, its rows stay unwritten, the launch returns, and
    every other system's forces equal the single-system path.  Clearing the injection
    restores a normal launch."""
    systems, params, pos, q, off = make_batch(4, 3000)
    b = B.rbe2d_batch_init(params, off)
    P_, Q_ = torch.as_tensor(pos, device="cuda"), torch.as_tensor(q, device="cuda")
    F = torch.full((off[-1], 3), float("nan"), dtype=torch.float32, device="cuda")
    bad, step = 2, 5
    with pytest.raises(B.RBE2DError) as ei:
        B.rbe2d_batch_set_wait(b, 0.0, -1)
    assert ei.value.code == B.RBE2D_EINVAL
    with pytest.raises(B.RBE2DError) as ei:
        B.rbe2d_batch_set_wait(b, 1e-3, len(systems))
    assert ei.value.code == B.RBE2D_EINVAL
    B.rbe2d_batch_set_wait(b, 1e-3, bad)
    B.rbe2d_batch_force(b, step, P_, Q_, B.RBE2D_KSPACE | B.RBE2D_IBC, F)
    with pytest.raises(B.RBE2DError) as ei:
        B.rbe2d_batch_sync_status(b)
    assert ei.value.code == B.RBE2D_ETIMEOUT
    Fb = F.cpu().numpy()
    assert np.all(np.isnan(Fb[off[bad]:off[bad + 1]]))  # the withheld system: left unwritten
    for s in range(len(systems)):
        if s == bad:
            continue
        sl = slice(off[s], off[s + 1])
        Fs, _, _, _ = single(params[s], pos[sl], q[sl], step)
        assert rel_l2(Fb[sl], Fs) < 1e-5, s
    # the status was cleared; without the injection the next launch is complete
    B.rbe2d_batch_set_wait(b, 2.0, -1)
    B.rbe2d_batch_force(b, step, P_, Q_, B.RBE2D_KSPACE | B.RBE2D_IBC, F)
    B.rbe2d_batch_sync_status(b)
    Fb = F.cpu().numpy()
    sl = slice(off[bad], off[bad + 1])
    Fs, _, _, _ = single(params[bad], pos[sl], q[sl], step)
    assert rel_l2(Fb[sl], Fs) < 1e-5
    B.rbe2d_batch_destroy(b)


def test_every_batched_variant_matches_the_single_system_path():
    """Each kernel variant the batch autotuner chooses from (register cap, FMA-pipe angles)
    and a small and a large chunk size give every system's forces within the FP32 bar of
    the single-system path; out-of-range choices are refused."""
    systems, params, pos, q, off = make_batch(6, 3000)
    b = B.rbe2d_batch_init(params, off)
    P_, Q_ = torch.as_tensor(pos, device="cuda"), torch.as_tensor(q, device="cuda")
    F = torch.empty((off[-1], 3), dtype=torch.float32, device="cuda")
    ref = [single(params[s], pos[off[s]:off[s + 1]], q[off[s]:off[s + 1]], 9)[0] for s in range(len(systems))]
    for variant in range(4):
        for sc, fc in ((256, 256), (2048, 1024)):
            B.rbe2d_batch_set_tuning(b, sc, fc, 152 * 4, variant)
            B.rbe2d_batch_force(b, 9, P_, Q_, B.RBE2D_KSPACE | B.RBE2D_IBC, F)
            B.rbe2d_batch_sync_status(b)
            Fb = F.cpu().numpy()
            for s in range(len(systems)):
                assert rel_l2(Fb[off[s]:off[s + 1]], ref[s]) < 1e-4, (variant, sc, fc, s)
    for bad in ((128, 256, 608, 0), (256, 256, 0, 0), (256, 256, 608, 4)):
        with pytest.raises(B.RBE2DError):
            B.rbe2d_batch_set_tuning(b, *bad)
    B.rbe2d_batch_destroy(b)
