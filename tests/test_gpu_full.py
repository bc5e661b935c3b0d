"""The full-size streamer (10 mm gap, 256 x 256 x 512 cells, 2 mm needle at
15.6 kV, photoionization) initialises and steps with its coupled solve: the
solve meets its tolerance, the field at the needle tip exceeds the background,
photoelectrons appear and the electron count stays sane."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2110_14494_gb300 import build
    build.build()


def test_full_size_streamer_steps():
    from paper_2110_14494_gb300 import PicContext
    wl = W.streamer_full()
    g = wl["grid"]
    mask = W.needle_mask(g, wl["needle_length"], wl["needle_radius"])
    ctx = PicContext(W.synthetic_air(), g, precision=32, capacity=30_000_000, seed=2110144950, dt=wl["dt"],
                     mask=mask, n_ppc=wl["n_ppc"], w_min=wl["w_min"], growth_trigger=wl["growth_trigger"],
                     particle_cap=20_000_000, sort_interval=20, coupled=True, v_lo=0.0, v_hi=wl["v_top"],
                     v_mask=wl["v_top"], poisson_rtol=1e-6, poisson_max_cycles=200, boundary=1, adaptive_dt=True,
                     photo_xi=wl["photo_xi"], photo_pq=wl["photo_pq"])
    w0 = wl["seed_n0"] * np.pi ** 1.5 * wl["seed_radius"] ** 3 / wl["n_initial"]
    n0 = ctx.seed_gaussian(wl["seed_n0"], wl["seed_radius"], wl["seed_center"], w0)
    assert 0.4e6 < n0 < 1.1e6   # the part of the seed inside the electrode is dropped
    photo = 0
    for _ in range(20):
        st = ctx.step(1, stats=True)
        assert st.poisson_rel_res <= 1e-6
        photo += st.n_photo
    assert 0.2 * n0 < st.n_end < 20 * n0
    assert photo > 0
    assert 0 < st.dt_last <= 2e-12
