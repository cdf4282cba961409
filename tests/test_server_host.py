"""Host-side logic of the serving API, without a GPU: argument checks,
"never admissible" requests (EBIT_EFULL) and unknown tickets.  No CUDA call
happens before the first admissible submission, so these run on the CPU."""
import pytest

from paper_2309_00338_gb300 import build


@pytest.fixture(scope="module")
def ebit():
    build.build_library()
    from paper_2309_00338_gb300 import ebit as E
    E.lib()
    return E


def test_budget_and_validation(ebit):
    s = ebit.ebit_server_create(64 << 20)  # 64 MiB
    try:
        big, keep = ebit.make_request(4096, [(0.5, 0.5, 0.1)], steps=5)
        with pytest.raises(ebit.EbitError) as e:
            ebit.ebit_submit(s, big)
        assert e.value.status == ebit.EBIT_EFULL
        # footprint estimate is monotone in n: a grid that fits the budget alone
        small_fp = ebit.ebit_footprint(64, 64, 1 / 64, ebit.EBIT_FP64)
        assert small_fp < 64 << 20
        for bad in (dict(n=0), dict(cfl=1.5), dict(cfl=0.0), dict(steps=-1), dict(field=9),
                    dict(field=ebit.EBIT_FIELD_VORTEX, period=0.0), dict(prec=7), dict(flags=8)):
            kw = dict(n=32, circles=[(0.5, 0.5, 0.2)], steps=3)
            kw.update(bad)
            r, keep = ebit.make_request(**kw)
            with pytest.raises(ebit.EbitError) as e:
                ebit.ebit_submit(s, r)
            assert e.value.status == ebit.EBIT_EINVAL, bad
        with pytest.raises(ebit.EbitError) as e:
            ebit.ebit_poll(s, 12345)
        assert e.value.status == ebit.EBIT_EINVAL
        with pytest.raises(ebit.EbitError) as e:
            ebit.ebit_cancel(s, 12345)
        assert e.value.status == ebit.EBIT_EINVAL
        assert ebit.lib().ebit_cancel(None, 1) == ebit.EBIT_EINVAL
        st = ebit.ebit_server_stats_get(s)
        assert st["queued"] == 0 and st["batch_steps"] == 0 and st["bytes_in_use"] == 0
    finally:
        ebit.ebit_server_destroy(s)


def test_create_rejects_zero_budget(ebit):
    import ctypes
    h = ctypes.c_void_p()
    assert ebit.lib().ebit_server_create(ctypes.byref(h), 0, None) == ebit.EBIT_EINVAL
