"""CPU checks of the C ABI: the library loads, exports every symbol include/epsr.h
declares, and rejects bad arguments on the host before touching the GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1904_08756_gb300 import epsr, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions(name="epsr.h"):
    src = open(os.path.join(ROOT, "include", name)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(epsr_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1904_08756_gb300 import build
    build.build()
    return epsr.lib()


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 25
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(epsr.EXPORTS) == names
    # the measurement probes live in their own library, not in the product one
    probe = header_functions("epsr_probe.h")
    assert sorted(epsr.PROBE_EXPORTS) == probe
    pl = epsr.probe_lib()
    for n in probe:
        assert hasattr(pl, n), n
        assert n not in names


def test_status_strings(lib):
    assert epsr.epsr_strerror(0) == "success"
    assert "timed out" in epsr.epsr_strerror(epsr.EPSR_ETIMEOUT)
    assert epsr.epsr_version() >= 10000


def _create(lib, desc, xyz, typ, ms):
    h = C.c_void_p()
    st = lib.epsr_box_create(C.byref(desc), xyz.ctypes.data, typ.ctypes.data, ms.ctypes.data,
                             None, C.byref(h))
    return st, h


def test_create_rejects_bad_input_on_host(lib):
    s = synth.water_box(10, seed=1, L_A=10.0)
    xyz = np.ascontiguousarray(s.xyz, np.int32)
    typ = np.ascontiguousarray(s.type, np.int32)
    ms = np.ascontiguousarray(s.mol_start, np.int64)
    bad = []
    d = epsr.box_desc(s); d.n_types = 0; bad.append((d, xyz, typ, ms))
    d = epsr.box_desc(s); d.n_bins = 0; bad.append((d, xyz, typ, ms))
    d = epsr.box_desc(s); d.move_kind = 7; bad.append((d, xyz, typ, ms))
    d = epsr.box_desc(s); d.temperature = -1; bad.append((d, xyz, typ, ms))
    d = epsr.box_desc(s); bad.append((d, xyz, typ + 5, ms))               # type out of range
    x2 = xyz.copy(); x2[3, 1] = s.L_fx; bad.append((epsr.box_desc(s), x2, typ, ms))
    m2 = ms.copy(); m2[2] = m2[1]; bad.append((epsr.box_desc(s), xyz, typ, m2))
    d = epsr.box_desc(s); d.move_kind = epsr.MOVE_ATOM; bad.append((d, xyz, typ, ms))
    for d, x, t, m in bad:
        st, h = _create(lib, d, x, t, m)
        assert st == epsr.EPSR_EINVAL and not h.value
        buf = C.create_string_buffer(256)
        assert lib.epsr_last_error_detail(buf, 256) == epsr.EPSR_EINVAL
        assert len(buf.value) > 0


def test_null_handles_are_rejected(lib):
    n = C.c_int64()
    assert lib.epsr_box_info(None, None, C.byref(n), None) == epsr.EPSR_EINVAL
    assert lib.epsr_box_destroy(None) == epsr.EPSR_OK
    assert lib.epsr_mc_set_batch(None, 4) == epsr.EPSR_EINVAL
    assert lib.epsr_sq_plan_destroy(None) == epsr.EPSR_OK
    assert lib.epsr_mc_set_cells(None, 0, 0) == epsr.EPSR_EINVAL
    assert lib.epsr_checkpoint_save(None, None, 0, None) == epsr.EPSR_EINVAL
    assert lib.epsr_checkpoint_load(None, None, 0, None) == epsr.EPSR_EINVAL
    assert lib.epsr_launch_count(None) == epsr.EPSR_EINVAL
    n0 = C.c_uint64()
    assert lib.epsr_launch_count(C.byref(n0)) == epsr.EPSR_OK


def test_flexible_descriptor_checked_on_host(lib):
    """Flexible molecules: the spring tables must be symmetric, finite and non-negative."""
    s = synth.flexible_water_box(10, seed=1, L_A=10.0)
    xyz = np.ascontiguousarray(s.xyz, np.int32)
    typ = np.ascontiguousarray(s.type, np.int32)
    ms = np.ascontiguousarray(s.mol_start, np.int64)
    M = epsr.MAX_TYPES
    bad = []
    d = epsr.box_desc(s); d.bond_k[0 * M + 1] = d.bond_k[1 * M + 0] + 1.0; bad.append(d)     # not symmetric
    d = epsr.box_desc(s); d.bond_k[0 * M + 1] = d.bond_k[1 * M + 0] = -1.0; bad.append(d)     # negative
    d = epsr.box_desc(s); d.bond_d[0 * M + 1] = d.bond_d[1 * M + 0] = float("nan"); bad.append(d)
    for d in bad:
        st, h = _create(lib, d, xyz, typ, ms)
        assert st == epsr.EPSR_EINVAL and not h.value


def test_histogram_buffers_checked_before_any_launch():
    """A histogram or g buffer that is too short, of the wrong type or on another device is
    refused by the binding before the library sees it (the kernels would write past it)."""
    torch = pytest.importorskip("torch")
    from paper_1904_08756_gb300 import epsr
    with pytest.raises(ValueError):
        epsr._hist_ptr(torch.zeros(5, dtype=torch.int64), 6)
    with pytest.raises(ValueError):
        epsr._hist_ptr(torch.zeros(10, dtype=torch.float32), 6)
    with pytest.raises(ValueError):
        epsr._g_ptr(torch.zeros(10, dtype=torch.float64), 6)
    with pytest.raises(ValueError):          # right length and type, but host memory
        epsr._hist_ptr(torch.zeros(10, dtype=torch.int64), 6)
