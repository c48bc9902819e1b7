"""Two steps per launch with 16-bit storage (FP16, BF16, block-int16).

A launch decodes the stored state once, performs two FP32 site updates per site and encodes the result once.
So it must equal, bit for bit, this emulation: decode the 16-bit state on the host (numpy), advance an FP32
handle two single steps from it, encode the FP32 result on the host with the storage format's rounding.  The
FP32 stepping is tied to the oracle by the other parity tests; the codecs here are written out independently
of the CUDA ones (round-to-nearest-even conversions, block exponent = floor(log2 max|v|) + 1 of each 4-site
group).  Sources act at both steps and receivers record at both; traces must match too.  The accuracy of the
16-bit forms against the oracle over 500 and 5000 steps is covered in test_gpu_parity.py."""
import numpy as np
import pytest

from paper_1108_2651_gb300 import lbem, workloads as W

pytestmark = pytest.mark.gpu

STORAGES = ["f16", "bf16", "i16b"]


def _f16_scale(p):
    """The power-of-two FP16 storage scale lbem_set_fields picks (largest |E|, |B|, |amplitude| -> about 2^7)."""
    m = 0.0
    for a in (p.E0, p.B0, p.src_amp):
        if a is not None and np.size(a):
            m = max(m, float(np.max(np.abs(np.asarray(a, np.float32)))))
    k = 0 if m <= 0 else 7 - int(np.ceil(np.log2(m)))
    return np.float32(2.0 ** max(-40, min(40, k)))


def _decode(st, raw, ex, scale):
    if st == "f16":
        return raw.view(np.float16).astype(np.float32) * np.float32(1.0 / scale)
    if st == "bf16":
        return (raw.astype(np.uint32) << 16).view(np.float32)
    e = np.repeat(ex.astype(np.int32), 4, axis=-1)
    f = np.where(e == -128, np.float32(0.0), np.ldexp(np.float32(1.0), e - 15).astype(np.float32)).astype(np.float32)
    return raw.view(np.int16).astype(np.float32) * f


def _encode(st, v, scale):
    """v: float32 [..., nx] with nx % 4 == 0; returns (raw uint16, exponents int8 or None)."""
    if st == "f16":
        return (v * scale).astype(np.float16).view(np.uint16), None
    if st == "bf16":
        u = v.view(np.uint32).astype(np.uint64)
        r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
        return r, None  # (no NaN in these states)
    blk = v.reshape(v.shape[:-1] + (v.shape[-1] // 4, 4))
    m = np.max(np.abs(blk), axis=-1)
    e = (((m.view(np.uint32) >> 23) & 0xFF).astype(np.int32) - 127 + 1)
    s = np.ldexp(np.float32(1.0), np.clip(15 - e, -126, 127)).astype(np.float32)
    q = np.clip(np.rint(blk * s[..., None]), -32767, 32767).astype(np.int32)
    big = ~(m < np.float32(2.0 ** 100))
    tiny = m < np.float32(2.0 ** -100)
    e = np.where(big, 127, np.where(tiny, -128, e))
    q = np.where(big[..., None], 32767, np.where(tiny[..., None], 0, q))
    return q.astype(np.int16).reshape(v.shape).view(np.uint16), e.astype(np.int8)


def _snapshot(s, st, shape):
    """Stored state as (raw [5][ny][pitch] uint16 or float32, exponents [5][ny][pitch/4] or None)."""
    import torch

    ny, nx = shape
    pitch = (nx + 31) // 32 * 32
    nb = lbem.lbem_info(s.h)[1]
    buf = torch.empty(nb, dtype=torch.uint8, device="cuda")
    lbem.lbem_save_state(s.h, buf)
    torch.cuda.synchronize()
    b = buf.cpu().numpy()
    if st == "f32":
        return b[: 5 * ny * pitch * 4].view(np.float32).reshape(5, ny, pitch), None
    raw = b[: 5 * ny * pitch * 2].view(np.uint16).reshape(5, ny, pitch)
    ex = b[5 * ny * pitch * 2:].view(np.int8).reshape(5, ny, pitch // 4) if st == "i16b" else None
    return raw, ex


def _problem(shape, seed, nsteps):
    eps, _ = W.random_medium(shape, seed)
    p = W.Problem("t16", 2, shape, eps, None, nsteps)
    p.E0, p.B0 = W.random_fields(shape, seed + 1, 0.3)
    p.E0[..., :2] = 0
    p.B0[..., 2] = 0
    n = int(np.prod(shape))
    rng = np.random.default_rng(seed + 2)
    p.src_site = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 3)])).astype(np.int64)
    p.src_comp = np.full(p.src_site.size, 2, np.int32)
    p.src_amp = rng.normal(0, 0.2, (p.src_site.size, nsteps))
    p.rec_site = np.unique(np.concatenate([[0, n // 2, n - 1], rng.integers(0, n, 5)])).astype(np.int64)
    p.rec_comp = np.array([2, 3, 4] * ((p.rec_site.size + 2) // 3), np.int32)[: p.rec_site.size]
    return p


@pytest.mark.parametrize("shape", [(1, 4), (17, 44), (33, 260), (6, 300), (130, 132), (64, 520)])
@pytest.mark.parametrize("st", STORAGES)
def test_two_step_16bit_equals_decode_two_fp32_steps_encode(lbem, st, shape):
    import torch

    ny, nx = shape
    nsteps = 9
    p = _problem(shape, 300 + nx, nsteps)
    scale = _f16_scale(p) if st == "f16" else np.float32(1.0)
    nshape = None
    for tile_shape in range(7):
        h16 = lbem.Solver(shape, storage=st)
        h16.set_problem(p)
        lbem.lbem_set_temporal_blocking(h16.h, 1, -1)
        h16.step(3)  # a non-trivial stored state at an odd time
        raw, ex = _snapshot(h16, st, shape)
        nshape = lbem.lbem_get_temporal_blocking(h16.h)[2]
        # emulation: decode, two FP32 steps (twice), encode after each pair
        h32 = lbem.Solver(shape)
        h32.set_problem(p)
        lbem.lbem_set_temporal_blocking(h32.h, 1, -1)
        exp_raw, exp_ex = raw, ex
        for pair in range(2):
            dec = _decode(st, exp_raw, exp_ex, scale)
            st32 = torch.from_numpy(np.ascontiguousarray(dec).view(np.uint8).ravel()).cuda()
            lbem.lbem_load_state(h32.h, st32, 3 + 2 * pair)
            h32.step(2)
            v, _x = _snapshot(h32, "f32", shape)
            v = np.ascontiguousarray(v[:, :, :nx])
            r, e = _encode(st, v, scale)
            exp_raw = np.zeros_like(raw)
            exp_raw[:, :, :nx] = r
            if st == "i16b":
                exp_ex = np.zeros_like(ex)
                exp_ex[:, :, : nx // 4] = e
        # the two-step kernel: two launches from the same stored state
        lbem.lbem_set_temporal_blocking(h16.h, 2, tile_shape)
        assert lbem.lbem_get_temporal_blocking(h16.h)[0] == 2
        h16.step(4)
        got_raw, got_ex = _snapshot(h16, st, shape)
        np.testing.assert_array_equal(got_raw[:, :, :nx], exp_raw[:, :, :nx], err_msg=f"{st} tile shape {tile_shape}")
        if st == "i16b":
            np.testing.assert_array_equal(got_ex[:, :, : nx // 4], exp_ex[:, :, : nx // 4])
        tr16 = h16.traces(p.rec_site.size).cpu().numpy()
        tr32 = h32.traces(p.rec_site.size).cpu().numpy()
        np.testing.assert_array_equal(tr16[:, 3:7], tr32[:, 3:7], err_msg=f"traces, {st} tile shape {tile_shape}")
        lbem.lbem_sync(h16.h)
        lbem.lbem_check_guards(h16.h)
        h16.close()
        h32.close()
    assert nshape == 7


def test_two_step_16bit_needs_nx_multiple_of_4_and_uniform_mu(lbem):
    import torch

    s = lbem.Solver((8, 30), storage="bf16")
    assert lbem.lbem_get_temporal_blocking(s.h)[0] == 1  # falls back to single steps
    s.close()
    s = lbem.Solver((8, 32), storage="bf16")
    assert lbem.lbem_get_temporal_blocking(s.h)[0] == 2
    lbem.lbem_set_medium(s.h, torch.ones(256, device="cuda"), torch.full((256,), 2.0, device="cuda"))
    assert lbem.lbem_get_temporal_blocking(s.h)[0] == 1  # a mu array (source term with grad ln mu): single steps
    s.close()
