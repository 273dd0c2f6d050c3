"""Checkpoint and resume (pm_save / pm_load): a run saved at a step
boundary and resumed in a fresh context gives the same bits as the
uninterrupted run, through the periodic and open phases, for the static
and diffusion gravities, with and without reordering by cell; a checkpoint
of another configuration, or a file that is not one, is refused."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1709_04703_gb300 import ics  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_04703_gb300 import build
    build.build()


N, BOX, A0, STEPS = 32, 6000.0, 0.2, 24


def _new(**kw):
    from paper_1709_04703_gb300.sim import Sim
    pos, mom, ids = ics.zeldovich(N, -1.5, 0.5, 6, A0, rms_disp=0.6)
    return Sim(pos, mom, ids, N, BOX, A0, 1.0, STEPS, **kw)


def _state(sim):
    st = sim.stats()
    p, m, i = sim.particles()
    lp, lm, li, la = sim.lightcone()
    return st, (p, m, i, lp, lm, li, la)


@pytest.mark.parametrize("kw", [dict(), dict(sort_every=5), dict(gravity="diffusion"),
                                dict(precision="fp32", rtol=1e-4),
                                dict(shrink="record", bc="periodic")])
@pytest.mark.parametrize("cut", [7, 15])
def test_resume_gives_the_same_bits(tmp_path, kw, cut):
    ref = _new(**kw)
    ref.step(STEPS)
    s_ref, a_ref = _state(ref)
    ref.close()
    first = _new(**kw)
    first.step(cut)
    path = tmp_path / "run.ckpt"
    first.save(path)
    first.close()
    second = _new(**kw)
    second.load(path)
    assert second.stats()["step"] == cut
    second.step(STEPS - cut)
    s_res, a_res = _state(second)
    second.close()
    for f in ("step", "n_active", "n_lightcone", "vcycles_total", "escaped", "particle_steps",
              "resid_last", "cube_side", "cube_lo"):
        assert s_res[f] == s_ref[f], f
    for u, v in zip(a_res, a_ref):
        np.testing.assert_array_equal(u, v)


def test_another_configuration_is_refused(tmp_path):
    from paper_1709_04703_gb300 import _lib as L
    a = _new()
    a.step(2)
    path = tmp_path / "a.ckpt"
    a.save(path)
    a.close()
    b = _new(rtol=1e-6)
    with pytest.raises(L.PmError) as e:
        b.load(path)
    assert e.value.code == L.PM_EINVAL
    junk = tmp_path / "junk.ckpt"
    junk.write_bytes(b"not a checkpoint" * 64)
    with pytest.raises(L.PmError) as e:
        b.load(junk)
    assert e.value.code in (L.PM_EINVAL, L.PM_EIO)
    with pytest.raises(L.PmError) as e:
        b.load(tmp_path / "missing.ckpt")
    assert e.value.code == L.PM_EIO
    b.step(1)   # the context is still usable
    b.close()


def test_corrupted_cube_is_refused(tmp_path):
    """A header whose active cube does not belong to its step (a truncated
    or edited file) is refused before anything is written to the device."""
    import ctypes as C
    from paper_1709_04703_gb300 import _lib as L

    class Head(C.Structure):   # the leading fields of the checkpoint header
        _fields_ = [("magic", C.c_char * 8), ("version", C.c_uint32),
                    ("header_bytes", C.c_uint32), ("cfg", L.PmConfig),
                    ("step", C.c_int32), ("cur", C.c_int32), ("n_sol", C.c_int32),
                    ("field_ready", C.c_int32), ("vc_prev", C.c_int32),
                    ("cube_valid", C.c_int32), ("lo", C.c_int32), ("s", C.c_int32),
                    ("periodic", C.c_int32)]

    a = _new()
    a.step(2)
    path = tmp_path / "a.ckpt"
    a.save(path)
    a.close()
    raw = bytearray(path.read_bytes())
    h = Head.from_buffer_copy(bytes(raw[:C.sizeof(Head)]))
    assert h.cube_valid == 1 and h.lo == 0 and h.s == N and h.periodic == 1
    b = _new()
    for lo, s, per, n_sol in ((8, 2 * N, 1, h.n_sol), (N, N, 0, h.n_sol), (-1, N, 1, h.n_sol),
                              (0, N, 7, h.n_sol), (0, N, 1, -3)):
        bad = Head.from_buffer_copy(bytes(raw[:C.sizeof(Head)]))
        bad.lo, bad.s, bad.periodic, bad.n_sol = lo, s, per, n_sol
        p = tmp_path / "bad.ckpt"
        p.write_bytes(bytes(bad) + bytes(raw[C.sizeof(Head):]))
        with pytest.raises(L.PmError) as e:
            b.load(p)
        assert e.value.code == L.PM_EINVAL, (lo, s, per, n_sol)
    b.load(path)           # the intact file still loads
    assert b.stats()["step"] == 2
    b.step(1)
    b.close()
