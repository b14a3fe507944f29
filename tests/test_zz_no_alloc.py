"""The allocation-free step entry point against the allocating one.

cavity_step_block_noalloc serves callers that must not call cudaMalloc
(code living inside another framework's caching allocator or a fixed
memory arena).  It runs the same fused step kernel over a block the caller
holds, with its reduction scratch in a fixed array inside the library.  This
test feeds it the state of a cavity handle, twice in a row, and checks its
output against cavity_step on the same handle.  The file is named so that
pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2006_02602_gb300 import build
    build.build()
    import paper_2006_02602_gb300 as m
    m.load_library()
    return torch, m


def _block_state(m, h):
    return np.stack([m.cavity_get_block_array(h, 0, f)[0] for f in range(5)])


def test_noalloc_matches_cavity_step_twice(env):
    torch, m = env
    n = (40, 36, 34)  # 2 x 5 x 3 tiles, ragged in x, y and z
    with m.Cavity(*n, seed=3, noise_amp=1e-3, Ra=1e5) as c:
        c.step(5)
        shape_full = (5, n[2] + 4, n[1] + 4, n[0] + 4)
        q_in = torch.zeros(shape_full, dtype=torch.float64, device="cuda")
        q_out = torch.zeros(shape_full, dtype=torch.float64, device="cuda")
        out6 = torch.zeros(6, dtype=torch.float64, device="cuda")
        # the handle's own transfers grow its staging buffer on first use: do
        # them once before the free-memory reading
        c.set_fields(c.fields())
        _block_state(m, c.h)
        torch.cuda.synchronize()
        free_before = None
        for call in range(2):
            # start from a state without a pending centre shift
            c.set_fields(c.fields())
            q_in.copy_(torch.from_numpy(_block_state(m, c.h)))
            q_out.zero_()
            _, _, dt = c.time
            m.cavity_step_block_noalloc(q_in.data_ptr(), q_out.data_ptr(), n, c.params, dt, 0.0,
                                        out6.data_ptr(), torch.cuda.current_stream().cuda_stream)
            torch.cuda.synchronize()
            if call == 0:
                # after the first call (which looks up the scratch address on
                # this device) free device memory must stay the same
                free_before = torch.cuda.mem_get_info()[0]
            got = q_out.cpu().numpy()
            res6 = out6.cpu().numpy()

            c.step(1)  # the allocating entry point on the same state
            ref = _block_state(m, c.h)
            inner = (slice(None), slice(2, -2), slice(2, -2), slice(2, -2))
            for f in range(5):
                a, b = got[inner][f], ref[inner][f]
                err = np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)
                assert err <= 1e-12, (call, f, err)
            assert np.allclose(res6[:5], c.residual, rtol=1e-12, atol=0), call
            assert res6[5] == pytest.approx(c.time[2], rel=1e-13), call
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free_before


def test_noalloc_rejects_blocks_beyond_its_scratch(env):
    torch, m = env
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    out6 = torch.zeros(6, dtype=torch.float64, device="cuda")
    p = m.cavity_default_params()
    with pytest.raises(m.CavityError) as e:
        m.cavity_step_block_noalloc(buf.data_ptr(), out6.data_ptr(), (600, 600, 600), p, 1e-6, 0.0,
                                    out6.data_ptr(), None)
    assert e.value.code == m.CAVITY_ERR_INVALID_ARG
    assert m.load_library().cavity_step_block_noalloc(None, None, 8, 8, 8, ctypes.byref(p), 1e-6, 0.0,
                                                      None, None) == m.CAVITY_ERR_INVALID_ARG
