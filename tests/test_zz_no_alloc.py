"""The allocation-free histogram entry point (for callers that may not allocate device
memory, e.g. plug-ins under a framework-owned allocator or real-time loops) against the
regular entry point, through the C ABI on the GPU. Collected last on purpose: it must
pass both alone in a fresh process (the first call sets the scratch address up) and
after every other test."""
import numpy as np
import pytest

from paper_1904_08756_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1904_08756_gb300 import epsr  # noqa: E402

DEV = torch.device("cuda:0")


def regular(system):
    box = epsr.Box(system)
    H = torch.zeros(box.hist_len, dtype=torch.int64, device=DEV)
    box.epsr_partial_gr(H)
    torch.cuda.synchronize()
    return H.cpu().numpy()


@pytest.mark.parametrize("make", [lambda: synth.water_box(400, seed=71),          # ragged tiles
                                  lambda: synth.silica_box(700, seed=72),
                                  lambda: synth.paper_water()])
def test_noalloc_matches_regular_on_two_calls(make):
    s = make()
    ref = regular(s)
    for _ in range(2):            # the scratch keeps the previous call's contents
        H = torch.zeros_like(torch.from_numpy(ref)).to(DEV)
        epsr.epsr_partial_gr_noalloc(s, H)
        torch.cuda.synchronize()
        assert np.array_equal(H.cpu().numpy(), ref)      # integer counts: bit-exact


def test_noalloc_rejects_too_many_atoms():
    s = synth.uniform_gas(epsr.NOALLOC_MAX_ATOMS + 1, 120.0, seed=3)
    H = torch.zeros(3 * s.n_bins, dtype=torch.int64, device=DEV)
    with pytest.raises(epsr.EpsrError) as ei:
        epsr.epsr_partial_gr_noalloc(s, H)
    assert ei.value.status == epsr.EPSR_EINVAL
    assert epsr.epsr_noalloc_scratch_bytes() > 0
