"""Host-side logic of the package that runs without a GPU."""
import numpy as np
import pytest

import oracle
import synth


def test_dlt_corner_parametrisation_roundtrip():
    """The refinement's corner parametrisation reproduces a camera's homography and its inverse."""
    torch = pytest.importorskip("torch")
    from paper_1810_03988_gb300.autograd import corners_of, homography_from_corners, image_corners, params_from_corners
    cfg = synth.config_refine(scale=0.25)
    for c in cfg.cameras:
        cr = torch.tensor(corners_of(c.H, c.width, c.height))
        H = homography_from_corners(image_corners(c.width, c.height), cr).numpy()
        np.testing.assert_allclose(H, c.H / c.H[2, 2], rtol=1e-9, atol=1e-9)
        A = oracle.invert_h(c.H)
        p = params_from_corners(cr[None], torch.ones(1, dtype=torch.float64), [(c.width, c.height)],
                                [A[2, 2]]).numpy()[0]
        np.testing.assert_allclose(p[:8], A.reshape(9)[:8], rtol=1e-8, atol=1e-10)
