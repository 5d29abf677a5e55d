"""vplbm_step_noalloc: the allocation-free stepping entry point.

It exists for callers that must not allocate device memory while they run
(a host application whose device memory belongs to another framework's
caching allocator, or a control loop with a fixed memory budget that forbids
cudaMalloc/cudaFree after start-up).  Here the test itself allocates the
caller-side buffers with torch; the entry point takes its scratch from a
static device array and allocates nothing.

The check: two calls in a row through the C ABI give the populations,
history records and body state of the regular vplbm_create / vplbm_step
path after the same number of steps, bit for bit: both run the same step
kernel at the same 128 x 2 block shape, so nothing may differ.  A third
call without a history buffer still advances the body state.  This file is
collected last so that a first-failure run has already run every other
test.
"""
import numpy as np
import pytest

import workloads as wl
from helpers import REC

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
STORE = {"f64": np.float64, "f32": np.float32, "f16": np.float16}


def _stored_to_full(raw: np.ndarray, nx: int, ny: int, precision: str) -> np.ndarray:
    n = nx * ny
    ps = (n + 127) // 128 * 128
    planes = raw.reshape(9, ps)[:, :n].astype(np.float64).reshape(9, ny, nx)
    return planes if precision == "f64" else planes + W[:, None, None]


def _problem(kind: str) -> dict:
    p = wl.oscillating_disk(nx=300, ny=160, diameter=24, x_c=80)
    if kind == "ellipse":
        p["body"] = dict(p["body"], shape="ellipse", radius_b=6.0, theta=0.3)
    elif kind == "free_fall":
        # a disk falling under gravity across the channel flow: the caller's
        # velocities feed the tail's RK4 from the first step on
        r = 12.0
        m = 1.5 * np.pi * r * r
        p["body"] = {"radius": r, "x": 80.0, "y": 100.0, "vx": 0.002, "vy": -0.004, "motion": "free",
                     "mass": m, "inertia": 0.5 * m * r * r, "f_ext": (0.0, -m * (1 - 1 / 1.5) * 2e-5, 0.0),
                     "dof_mask": 7, "u_ref": 0.04, "d_ref": 2 * r}
    return p


def _caller_buffers(lat, body, cap, dev):
    import torch
    import paper_1905_05110_gb300 as vp
    sizes = vp.vplbm_buffer_sizes_for(lat, body, cap)
    pops = [torch.zeros(int(sizes.populations), dtype=torch.uint8, device=dev) for _ in range(2)]
    state = torch.zeros(64, dtype=torch.uint8, device=dev)
    return sizes, pops, state


def _state_bytes(b: dict) -> np.ndarray:
    import paper_1905_05110_gb300 as vp
    s = vp.BodyState()
    s.q[0], s.q[1], s.q[2] = b["x"], b["y"], b.get("theta", 0.0)
    s.v[0], s.v[1], s.v[2] = b.get("vx", 0.0), b.get("vy", 0.0), b.get("omega", 0.0)
    s.step = 0
    return np.frombuffer(bytes(s), dtype=np.uint8).copy()


@pytest.mark.parametrize("precision,kind", [("f32", "disk"), ("f64", "disk"), ("f16", "disk"),
                                            ("f32", "ellipse"), ("f32", "free_fall")])
def test_noalloc_two_calls_match_regular_step(gpu_library, precision, kind):
    import torch
    import paper_1905_05110_gb300 as vp

    p = _problem(kind)
    nx, ny = p["nx"], p["ny"]
    cap = 128
    ref = vp.Simulation(p, precision=precision, history_capacity=cap)
    ref.set_launch("scalar", 128, 2)   # the kernel and shape the no-alloc path runs
    ref.init_from_problem()

    lat = vp.lattice_desc(p, precision)
    body = vp.body_desc(p["body"])
    dev = torch.device("cuda")
    sizes, pops, state = _caller_buffers(lat, body, cap, dev)
    nbytes = int(sizes.populations)
    # caller-owned buffers: the initial state is the regular path's state 0
    src = ref._tensors["f0"]
    off = (-src.data_ptr()) % 256
    pops[0].copy_(src[off:off + nbytes])
    sb = _state_bytes(p["body"])
    state_dev = state[:sb.size]
    state_dev.copy_(torch.from_numpy(sb))
    hist_dev = torch.zeros(cap * 16, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream().cuda_stream

    def call(nsteps, cur, hist=True):
        vp.vplbm_step_noalloc(lat, body, [pops[cur].data_ptr(), pops[cur ^ 1].data_ptr()],
                              state_dev.data_ptr(), hist_dev.data_ptr() if hist else None, cap, nsteps, stream)
        torch.cuda.synchronize()
        return cur ^ (nsteps & 1)

    def body_state():
        return vp.BodyState.from_buffer_copy(state_dev.cpu().numpy().tobytes())

    cur = 0
    done = 0
    for nsteps in (40, 23):
        cur = call(nsteps, cur)
        done += nsteps
        ref.step(nsteps)
        raw = pops[cur].cpu().numpy().view(STORE[precision])
        assert np.array_equal(_stored_to_full(raw, nx, ny, precision), ref.populations())
        st = body_state()
        assert st.step == done and st.error == 0
        q_ref, v_ref = ref.body_state()
        assert np.array_equal(list(st.q), q_ref) and np.array_equal(list(st.v), v_ref)
        h_new = hist_dev.cpu().numpy().reshape(cap, 16)[:done]
        assert np.array_equal(h_new, ref.history(0, done))

    # a call without a history buffer still advances the body state, and
    # leaves the caller's history ring untouched
    h_before = hist_dev.clone()
    cur = call(9, cur, hist=False)
    ref.step(9)
    st = body_state()
    q_ref, v_ref = ref.body_state()
    assert st.step == done + 9 and st.error == 0
    assert np.array_equal(list(st.q), q_ref) and np.array_equal(list(st.v), v_ref)
    assert torch.equal(hist_dev, h_before)
    raw = pops[cur].cpu().numpy().view(STORE[precision])
    assert np.array_equal(_stored_to_full(raw, nx, ny, precision), ref.populations())
    if kind == "free_fall":
        assert st.q[1] < p["body"]["y"] and st.v[1] != p["body"]["vy"]
    assert np.array_equal(ref.history(done, 9)[:, REC["t"]], np.arange(done, done + 9, dtype=np.float64))
    ref.close()


def test_noalloc_rejects_what_it_cannot_hold(gpu_library):
    # Every call gets real device buffers of the sizes vplbm_buffer_sizes_for
    # gives, so that no case has a path to a fault even if a host check
    # moved: the entry point refuses each before any device work.
    import torch
    import paper_1905_05110_gb300 as vp

    dev = torch.device("cuda")

    def refused(p, precision="f32", shift=(0, 0, 0, 0), hist=False):
        lat = vp.lattice_desc(p, precision)
        body = vp.body_desc(p["body"])
        _, pops, state = _caller_buffers(lat, body, 4, dev)
        h = torch.zeros(4 * 16 + 1, dtype=torch.float64, device=dev)
        ptrs = [pops[0].data_ptr() + shift[0], pops[1].data_ptr() + shift[1]]
        with pytest.raises(vp.VplbmError) as ei:
            vp.vplbm_step_noalloc(lat, body, ptrs, state.data_ptr() + shift[2],
                                  h.data_ptr() + shift[3] if hist else None, 4, 1, 0)
        torch.cuda.synchronize()
        return ei.value

    # a disk of radius 900 on 2048 x 2048 meets about 16 x 900 tiles of the
    # 128 x 2 blocks, far beyond the 4096 slots of the static scratch (on a
    # lattice of at most 4096 such tiles nothing can exceed them)
    big = wl.oscillating_disk(nx=2048, ny=2048, diameter=1800, x_c=1024)
    big["body"] = dict(big["body"], y=1024.0)
    e = refused(big)
    assert e.status == 7 and "reduction slots" in str(e)
    e = refused(wl.channel_fixed_disk())
    assert e.status == 6
    conv = wl.oscillating_disk(nx=256, ny=128, diameter=16, x_c=60)
    conv["bc"]["east"] = {"kind": "convective", "u": (0.04, 0.0)}
    e = refused(conv)
    assert e.status == 6 and "outlet" in str(e)
    small = wl.oscillating_disk(nx=96, ny=48, diameter=10, x_c=30)
    for precision, shift, msg in (("f32", (2, 0, 0, 0), "element size"), ("f64", (0, 4, 0, 0), "element size"),
                                  ("f16", (1, 0, 0, 0), "element size"), ("f32", (0, 0, 4, 0), "8-byte"),
                                  ("f32", (0, 0, 0, 4), "8-byte")):
        e = refused(small, precision, shift, hist=True)
        assert e.status == 1 and msg in str(e), (precision, shift)
