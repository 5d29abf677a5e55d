"""vplbm_step_noalloc: the allocation-free stepping entry point.

It exists for callers that must not allocate device memory while they run
(a host application whose device memory belongs to another framework's
caching allocator, or a control loop with a fixed memory budget that forbids
cudaMalloc/cudaFree after start-up).  Here the test itself allocates the
caller-side buffers with torch; the entry point takes its scratch from a
static device array and allocates nothing.

The check: two calls in a row through the C ABI give the same populations,
history and body state, within the parity tolerances used by the other
tests, as the regular vplbm_create / vplbm_step path after the same number
of steps.  This file is collected last so that a first-failure run has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import workloads as wl
from helpers import REC, dev_err, rel_err

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
RUN_TOL = {"f64": 1e-12, "f32": 1e-4}
ELEM = {"f64": (8, np.float64), "f32": (4, np.float32)}


def _stored_to_full(raw: np.ndarray, nx: int, ny: int, precision: str) -> np.ndarray:
    n = nx * ny
    ps = (n + 127) // 128 * 128
    planes = raw.reshape(9, ps)[:, :n].astype(np.float64).reshape(9, ny, nx)
    return planes if precision == "f64" else planes + W[:, None, None]


@pytest.mark.parametrize("precision,shape", [("f32", "disk"), ("f64", "disk"), ("f32", "ellipse")])
def test_noalloc_two_calls_match_regular_step(gpu_library, precision, shape):
    import torch
    import paper_1905_05110_gb300 as vp

    p = wl.oscillating_disk(nx=300, ny=160, diameter=24, x_c=80)
    if shape == "ellipse":
        p["body"] = dict(p["body"], shape="ellipse", radius_b=6.0, theta=0.3)
    nx, ny = p["nx"], p["ny"]
    n1, n2 = 40, 23
    cap = 128
    ref = vp.Simulation(p, precision=precision, history_capacity=cap)
    ref.set_launch("scalar", 128, 2)   # the kernel and shape the no-alloc path runs
    ref.init_from_problem()

    lat = vp.lattice_desc(p, precision)
    body = vp.body_desc(p["body"])
    sizes = vp.vplbm_buffer_sizes_for(lat, body, cap)
    nbytes = int(sizes.populations)
    dev = torch.device("cuda")
    # caller-owned buffers: the initial state is the regular path's state 0
    src = ref._tensors["f0"]
    off = (-src.data_ptr()) % 256
    pops = [torch.empty(nbytes, dtype=torch.uint8, device=dev) for _ in range(2)]
    pops[0].copy_(src[off:off + nbytes])
    state = vp.BodyState()
    b = p["body"]
    state.q[0], state.q[1], state.q[2] = b["x"], b["y"], b.get("theta", 0.0)
    state.v[0], state.v[1], state.v[2] = b.get("vx", 0.0), b.get("vy", 0.0), b.get("omega", 0.0)
    state.step = 0
    state_dev = torch.from_numpy(np.frombuffer(bytes(state), dtype=np.uint8).copy()).to(dev)
    hist_dev = torch.zeros(cap * 16, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream

    def call(nsteps, cur):
        vp.vplbm_step_noalloc(lat, body, [pops[cur].data_ptr(), pops[cur ^ 1].data_ptr()],
                              state_dev.data_ptr(), hist_dev.data_ptr(), cap, nsteps, stream)
        torch.cuda.synchronize()
        return cur ^ (nsteps & 1)

    cur = 0
    done = 0
    for nsteps in (n1, n2):
        cur = call(nsteps, cur)
        done += nsteps
        ref.step(nsteps)
        f_ref = ref.populations()
        raw = pops[cur].cpu().numpy().view(ELEM[precision][1])
        f_new = _stored_to_full(raw, nx, ny, precision)
        assert dev_err(f_new, f_ref) < RUN_TOL[precision]
        st = vp.BodyState.from_buffer_copy(state_dev.cpu().numpy().tobytes())
        assert st.step == done and st.error == 0
        q_ref, v_ref = ref.body_state()
        assert np.allclose(list(st.q), q_ref, rtol=0, atol=1e-9)
        assert np.allclose(list(st.v), v_ref, rtol=0, atol=1e-12)
        h_new = hist_dev.cpu().numpy().reshape(cap, 16)[:done]
        h_ref = ref.history(0, done)
        assert np.array_equal(h_new[:, REC["t"]], h_ref[:, REC["t"]])
        for key in ("fx", "fy", "fpen_x", "fpen_y"):
            assert rel_err(h_new[:, REC[key]], h_ref[:, REC[key]]) < (1e-10 if precision == "f64" else 1e-3)
    ref.close()


def test_noalloc_rejects_what_it_cannot_hold(gpu_library):
    import paper_1905_05110_gb300 as vp

    big = wl.oscillating_disk(nx=4096, ny=4096, diameter=1200, x_c=2048)
    with pytest.raises(vp.VplbmError) as ei:
        vp.vplbm_step_noalloc(vp.lattice_desc(big, "f32"), vp.body_desc(big["body"]), [1 << 20, 1 << 21],
                              1 << 22, None, 0, 1, 0)
    assert ei.value.status == 7 and "reduction slots" in str(ei.value)
    prof = wl.channel_fixed_disk()
    with pytest.raises(vp.VplbmError) as ei:
        vp.vplbm_step_noalloc(vp.lattice_desc(prof, "f32"), vp.body_desc(prof["body"]), [1 << 20, 1 << 21],
                              1 << 22, None, 0, 1, 0)
    assert ei.value.status == 6
    conv = wl.oscillating_disk(nx=256, ny=128, diameter=16, x_c=60)
    conv["bc"]["east"] = {"kind": "convective", "u": (0.04, 0.0)}
    with pytest.raises(vp.VplbmError) as ei:
        vp.vplbm_step_noalloc(vp.lattice_desc(conv, "f32"), vp.body_desc(conv["body"]), [1 << 20, 1 << 21],
                              1 << 22, None, 0, 1, 0)
    assert ei.value.status == 6 and "outlet" in str(ei.value)
