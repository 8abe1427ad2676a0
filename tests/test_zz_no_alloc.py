"""pss_nls_invariants_static: the NLS mass and energy computed with the
library's static scratch array instead of allocated memory.

This entry point serves callers that cannot call cudaMalloc (device memory
owned by another allocator or a fixed budget, or loops where an allocation
and the synchronisation it may cause are not acceptable).  Its results must
agree with pss_conserved_quantities, the grid-based entry point, and two
calls in a row must not see each other's leftovers in the shared array.
This file is collected last so that a stop at its first failure has already
run every other test.
"""
import math

import numpy as np
import pytest

import synthetic as S

pytestmark = pytest.mark.gpu

L = 20 * math.pi
# the tolerances of the NLS invariant tests: FP64 to rounding, FP32 at the
# mass-drift bound
TOL = {"fp64": 1e-12, "fp32": 1e-6}


def _device_fields(lib, g, precision, cuda_device):
    """psi (physical) and its forward 2D DFT, both on the device."""
    import torch
    cdt = torch.complex64 if precision == "fp32" else torch.complex128
    psi = torch.empty((g.batch, g.ny, g.nx), dtype=cdt, device=cuda_device)
    g.get_state_device(psi)
    hat = psi.clone()
    prec = lib.PSS_FP32 if precision == "fp32" else lib.PSS_FP64
    lib.pss_fft2d(hat.data_ptr(), g.nx, g.ny, g.batch, prec, -1,
                  torch.cuda.current_stream().cuda_stream)
    return psi, hat, prec


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_invariants_match_grid_entry_point_twice(lib, orc, cuda_device, precision):
    import torch
    # two calls in a row that differ in grid size, batch and data: the first
    # (256^2, 8 fields, amplitudes scaled by 3) fills more of the shared
    # scratch than the second (16^2, 1 field) reads, so a partial sum the
    # second call failed to rewrite, or read from the wrong place, would
    # carry the first call's much larger values into its result
    cases = ((256, 8, S.SEED_BASE, 3.0), (16, 1, S.SEED_BASE + 77, 1.0))
    expect, calls, oracle_ref = [], [], []
    for n, batch, seed, amp in cases:
        fields = amp * S.nls_gaussian(n, seed=seed, batch=batch)
        g = lib.Grid("nls", n, precision, batch=batch, lx=L, ly=L, dt=1e-3)
        g.set_state(fields)
        expect.append(g.conserved())  # existing entry point: mass, energy per field
        psi, hat, prec = _device_fields(lib, g, precision, cuda_device)
        # the FP64 oracle on the same fields as the library holds them
        oracle_ref.append(np.array([orc.nls_invariants(f, L, L) for f in psi.cpu().numpy()]))
        out = torch.full((2 * batch,), float("nan"), dtype=torch.float64, device=cuda_device)
        lib.pss_nls_invariants_static(psi.data_ptr(), hat.data_ptr(), n, n, batch, L, L, 1.0,
                                      prec, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        calls.append(out.cpu().numpy().reshape(batch, 2))
        g.close()
    for got, ref, orf in zip(calls, expect, oracle_ref):
        assert np.all(np.isfinite(got))
        assert np.max(np.abs(got - ref) / np.abs(ref)) <= TOL[precision]
        assert np.max(np.abs(got - orf) / np.abs(orf)) <= TOL[precision]


def test_static_invariants_reject_batch_beyond_scratch(lib, cuda_device):
    import torch
    n, batch = 16, 65
    x = torch.zeros((batch, n, n), dtype=torch.complex64, device=cuda_device)
    out = torch.zeros(2 * batch, dtype=torch.float64, device=cuda_device)
    with pytest.raises(lib.PssError) as e:
        lib.pss_nls_invariants_static(x.data_ptr(), x.data_ptr(), n, n, batch, L, L, 1.0,
                                      lib.PSS_FP32, out.data_ptr())
    assert e.value.code == lib.PSS_E_ARG
    assert "64" in lib.pss_last_error(None)
