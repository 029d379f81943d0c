"""Frame streams (hrm_filter2d_video): every frame's median equals the oracle
and the single-image call, whatever topology the previous frame left."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hrm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1105_3829_gb300 import hrm as h
    h.lib()
    return h


@pytest.mark.parametrize("r", [3, 9, 20])
def test_frames_match_oracle_and_single_calls(hrm, oracle, r):
    from paper_1105_3829_gb300 import inputs
    topo = hrm.Topology()
    for f, frame in enumerate(inputs.video_frames(4, 150, 270, drift=6, seed=100 + r)):
        src = torch.from_numpy(frame).cuda()
        got = hrm.filter2d_video(src, r, topo)
        single = hrm.filter2d(src, r)
        hrm.device_status()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), single.cpu().numpy())
        if f in (0, 3):
            np.testing.assert_array_equal(got.cpu().numpy(), oracle.median2d(frame, r))
    topo.close()


def test_dtype_change_and_unrelated_frames(hrm, oracle):
    """A u8 frame after u16 frames, then a u16 frame unlike the previous ones:
    the stale estimate only costs speed."""
    from paper_1105_3829_gb300 import inputs
    topo = hrm.Topology()
    frames = [next(inputs.video_frames(1, 120, 200, seed=5)),
              np.random.default_rng(1).integers(0, 256, size=(90, 130)).astype(np.uint8),
              inputs.xray12_u16(120, 200, seed=9),
              np.full((64, 64), 65535, np.uint16)]
    for frame in frames:
        src = torch.from_numpy(frame).cuda()
        got = hrm.filter2d_video(src, 12, topo)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got.cpu().numpy(), oracle.median2d(frame, 12))
    topo.close()
