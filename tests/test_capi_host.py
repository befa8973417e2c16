"""CPU-only checks of the C-ABI library: it builds for sm_103a, loads, exports
every entry point include/tx16.h declares, and its host-only logic (argument
checking, block counts, PSNR) behaves -- no compute call needs a GPU here."""
import ctypes
import math
import os
import re

import pytest

from oracle import tx16_oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1606_07414_gb300 import build, tx16

    build.build()
    return tx16.load()


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(tx16_[a-z0-9_]+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared_symbols()
    assert {"tx16_forward", "tx16_quantise", "tx16_inverse", "tx16_codec_batch"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_status_strings(lib):
    from paper_1606_07414_gb300 import tx16

    assert tx16.status_str(0) == "ok"
    assert tx16.status_str(1) == "invalid argument"
    assert tx16.status_str(99) == "unknown status"


def _img(w, h, pitch=None, bits=8, ptr=0x10000):
    from paper_1606_07414_gb300 import tx16

    esz = 1 if bits == 8 else 2
    return tx16.tx16_image(ptr, w, h, pitch if pitch is not None else w * esz, bits)


def test_image_blocks_and_validation(lib):
    f = lib.tx16_image_blocks
    assert f(ctypes.byref(_img(512, 512))) == 1024
    assert f(ctypes.byref(_img(1920, 1088))) == 8160
    assert f(ctypes.byref(_img(3840, 2160, bits=10))) == 32400
    for bad in (_img(500, 512), _img(512, 0), _img(32, 32, pitch=40), _img(32, 32, pitch=16),
                _img(32, 32, bits=7), _img(32, 32, bits=13), _img(32, 32, ptr=0x10008),
                _img(32, 32, ptr=0), _img(32, 32, bits=10, pitch=48)):
        assert f(ctypes.byref(bad)) == -1


def test_argument_errors_launch_nothing(lib):
    """Invalid arguments return TX16_EINVAL before touching CUDA (so this runs
    without a GPU)."""
    from paper_1606_07414_gb300 import tx16

    good = (tx16.tx16_image * 1)(_img(32, 32))
    bad = (tx16.tx16_image * 1)(_img(30, 32))
    qp = (tx16.tx16_qparams * 1)(tx16.tx16_qparams(8.0, 16))
    qbad = (tx16.tx16_qparams * 1)(tx16.tx16_qparams(8.0, 0))
    qbad2 = (tx16.tx16_qparams * 1)(tx16.tx16_qparams(8.0, 257))
    qnan = (tx16.tx16_qparams * 1)(tx16.tx16_qparams(float("nan"), 16))
    dev = ctypes.c_void_p(0x20000)
    E = tx16.TX16_EINVAL
    assert lib.tx16_forward(bad, 1, dev, None) == E
    assert lib.tx16_forward(good, -1, dev, None) == E
    assert lib.tx16_forward(good, 1, None, None) == E
    assert lib.tx16_forward(good, 1, ctypes.c_void_p(0x20004), None) == E
    assert lib.tx16_codec_batch(good, None, 1, qbad, None, None, None) == E
    assert lib.tx16_codec_batch(good, None, 1, qbad2, None, None, None) == E
    assert lib.tx16_codec_batch(good, None, 1, qnan, None, None, None) == E
    assert lib.tx16_codec_batch(bad, None, 1, qp, None, None, None) == E
    other = (tx16.tx16_image * 1)(_img(48, 32))
    assert lib.tx16_codec_batch(good, other, 1, qp, None, None, None) == E
    assert lib.tx16_inverse(dev, bad, 1, qp, None) == E
    assert lib.tx16_inverse(dev, good, 1, qbad, None) == E
    assert lib.tx16_sse(good, other, 1, dev, None) == E
    assert lib.tx16_quantise(dev, 4, tx16.tx16_qparams(8.0, 0), dev, None) == E
    assert lib.tx16_quantise(dev, -1, tx16.tx16_qparams(8.0, 4), dev, None) == E
    # empty batches are valid no-ops
    assert lib.tx16_forward(good, 0, dev, None) == tx16.TX16_OK
    assert lib.tx16_quantise(dev, 0, tx16.tx16_qparams(8.0, 4), dev, None) == tx16.TX16_OK


def test_psnr_matches_oracle(lib):
    from paper_1606_07414_gb300 import tx16

    imgs = [_img(512, 512), _img(64, 32, bits=10), _img(16, 16)]
    sse = [123456, 2048, 0]
    got = tx16.tx16_psnr(sse, imgs)
    want = [O.psnr(123456, 512, 512, 8), O.psnr(2048, 32, 64, 10), math.inf]
    for g, w in zip(got, want):
        assert g == pytest.approx(w, rel=1e-15) if math.isfinite(w) else g == w


def test_serve_create_rejects_malformed_config_before_any_device_call(lib):
    import ctypes

    h = ctypes.c_void_p()
    for bad in (b"{", b"[1]", b'{"streams": }', b'{"streams" 3}', b'{streams: 3}'):
        assert lib.tx16_serve_create(bad, ctypes.byref(h)) == 1  # TX16_EINVAL


def test_new_entry_points_reject_bad_arguments_before_any_device_call(lib):
    """tx16_codec_any_size, tx16_ssim, tx16_codec_mixed and tx16_zonal_sweep
    check their arguments on the host and launch nothing on error."""
    from paper_1606_07414_gb300 import tx16

    E = tx16.TX16_EINVAL
    dev = ctypes.c_void_p(0x20000)
    qp = (tx16.tx16_qparams * 1)(tx16.tx16_qparams(8.0, 16))
    # any size: sides need not be multiples of 16, but pitch rules hold
    assert lib.tx16_codec_any_size((tx16.tx16_image * 1)(_img(37, 50, pitch=40)), None, 1, qp, None, None) == E
    assert lib.tx16_codec_any_size((tx16.tx16_image * 1)(_img(37, 50, pitch=32)), None, 1, qp, None, None) == E
    assert lib.tx16_codec_any_size((tx16.tx16_image * 1)(_img(0, 50, pitch=48)), None, 1, qp, None, None) == E
    assert lib.tx16_codec_any_size((tx16.tx16_image * 1)(_img(37, 50, pitch=48)),
                                   (tx16.tx16_image * 1)(_img(36, 50, pitch=48)), 1, qp, None, None) == E
    assert lib.tx16_codec_any_size((tx16.tx16_image * 1)(_img(37, 50, pitch=48)), None, 1, qp,
                                   ctypes.c_void_p(0x20004), None) == E
    # SSIM: both sides at least 11, equal shapes and depths
    a = (tx16.tx16_image * 1)(_img(10, 32, pitch=16))
    b = (tx16.tx16_image * 1)(_img(32, 32))
    c = (tx16.tx16_image * 1)(_img(32, 32, bits=10, pitch=64))
    assert lib.tx16_ssim(a, a, 1, dev, None, None) == E
    assert lib.tx16_ssim(b, c, 1, dev, None, None) == E
    assert lib.tx16_ssim(b, b, 1, None, None, None) == E
    assert lib.tx16_ssim(b, b, 1, ctypes.c_void_p(0x20004), None, None) == E
    # mixed tiling: r16 in 1..256, r8 in 1..64, mode 0..2, finite q
    good = (tx16.tx16_image * 1)(_img(32, 32))
    for q, r16, r8, mode in [(8.0, 0, 4, 0), (8.0, 16, 0, 0), (8.0, 16, 65, 0), (8.0, 16, 4, 3),
                             (float("inf"), 16, 4, 0)]:
        m = (tx16.tx16_mixed_qparams * 1)(tx16.tx16_mixed_qparams(q, r16, r8, mode))
        assert lib.tx16_codec_mixed(good, None, 1, ctypes.cast(m, ctypes.c_void_p), None, None, None) == E
    m = (tx16.tx16_mixed_qparams * 1)(tx16.tx16_mixed_qparams(8.0, 16, 4, 0))
    assert lib.tx16_codec_mixed((tx16.tx16_image * 1)(_img(30, 32)), None, 1,
                                ctypes.cast(m, ctypes.c_void_p), None, None, None) == E
    # zonal sweep: 1 <= nr <= 16, r in 1..256
    rl = (ctypes.c_int32 * 17)(*([16] * 17))
    assert lib.tx16_zonal_sweep(good, 1, rl, 17, dev, None) == E
    assert lib.tx16_zonal_sweep(good, 1, (ctypes.c_int32 * 1)(0), 1, dev, None) == E
    assert lib.tx16_zonal_sweep(good, 1, (ctypes.c_int32 * 1)(257), 1, dev, None) == E
    # empty batches are valid no-ops
    assert lib.tx16_codec_any_size(good, None, 0, qp, None, None) == tx16.TX16_OK
    assert lib.tx16_codec_mixed(good, None, 0, ctypes.cast(m, ctypes.c_void_p), None, None, None) == tx16.TX16_OK


def test_static_entry_point_rejects_bad_arguments_before_any_device_call(lib):
    """tx16_codec_batch_static checks its arguments on the host: the batch size
    against its fixed array, alignment of the level and error buffers, and
    every descriptor and quantiser, launching nothing on error."""
    from paper_1606_07414_gb300 import tx16

    E = tx16.TX16_EINVAL
    qp1 = (tx16.tx16_qparams * 1)(tx16.tx16_qparams(8.0, 16))
    good = (tx16.tx16_image * 1)(_img(32, 32))
    f = lib.tx16_codec_batch_static
    assert f(good, None, -1, qp1, None, None, None) == E
    big = tx16.TX16_STATIC_MAX_IMAGES + 1
    assert f((tx16.tx16_image * big)(*[_img(32, 32)] * big), None, big,
             (tx16.tx16_qparams * big)(*[tx16.tx16_qparams(8.0, 16)] * big), None, None, None) == E
    assert f(None, None, 1, qp1, None, None, None) == E
    assert f(good, None, 1, None, None, None, None) == E
    assert f(good, None, 1, qp1, ctypes.c_void_p(0x20004), None, None) == E  # sse not 8-byte aligned
    assert f(good, None, 1, qp1, None, ctypes.c_void_p(0x20008), None) == E  # levels not 16-byte aligned
    assert f((tx16.tx16_image * 1)(_img(30, 32)), None, 1, qp1, None, None, None) == E
    assert f(good, (tx16.tx16_image * 1)(_img(32, 48)), 1, qp1, None, None, None) == E
    assert f(good, (tx16.tx16_image * 1)(_img(32, 32, bits=10, pitch=64)), 1, qp1, None, None, None) == E
    for q, r in [(8.0, 0), (8.0, 257), (float("inf"), 16), (float("nan"), 16)]:
        assert f(good, None, 1, (tx16.tx16_qparams * 1)(tx16.tx16_qparams(q, r)), None, None, None) == E
    assert f(good, None, 0, qp1, None, None, None) == tx16.TX16_OK  # empty batch: a no-op


def test_build_refuses_flush_to_zero_flags(monkeypatch):
    """The fused kernels' sample rounding goes through subnormal binary32
    values, so extra nvcc flags that flush them are refused before compiling."""
    from paper_1606_07414_gb300 import build

    for bad in ("-ftz=true", "--use_fast_math", "-O3 -use_fast_math"):
        monkeypatch.setenv("TX16_NVCC_FLAGS", bad)
        with pytest.raises(ValueError):
            build.extra_flags()
    monkeypatch.setenv("TX16_NVCC_FLAGS", "-DTX16_BT_MINCTAS_B=3 -ftz=false")
    assert build.extra_flags() == ["-DTX16_BT_MINCTAS_B=3", "-ftz=false"]


def test_class_heights_are_the_zigzag_column_heights():
    """The one-block-per-thread kernel prunes each column pair to the taller
    column's height in Z_rmax of its class (compile-time tables in the kernel
    source): they must be the oracle's zig-zag column heights, so that no
    kept coefficient of any r <= r_max is dropped (Sec. 3.1 zonal scan)."""
    src = open(os.path.join(ROOT, "paper_1606_07414_gb300", "csrc", "tx16_fused_bt.cuh")).read()
    found = re.findall(r"struct BtClass<(\d)> \{\s*static constexpr int kRmax = (\d+), V = (\d+), U = (\d+);"
                       r"\s*static constexpr int H\[\d+\] = \{([^}]*)\};", src)
    assert len(found) == 6
    for c, rmax, V, U, H in found:
        rmax, V, U = int(rmax), int(V), int(U)
        H = [int(x) for x in H.split(",")]
        m = O.zonal_mask(rmax)
        colh = [int(m[:, v].sum()) for v in range(16)]
        assert V == max(v + 1 for v in range(16) if colh[v] > 0), c
        assert U == max(colh), c
        assert H == [max(colh[2 * p], colh[2 * p + 1]) for p in range(V // 2)], c


def test_mixed_8x8_class_heights_are_the_zigzag_column_heights():
    """The mixed-tiling kernel prunes each 8x8 column to its height in the
    8x8 zig-zag zone Z_rmax of its class; the dispatcher's copy of the tables
    must agree, and both must be the oracle's 8x8 zig-zag column heights."""
    src = open(os.path.join(ROOT, "paper_1606_07414_gb300", "csrc", "tx16_mixed_bt.cuh")).read()
    found = re.findall(r"struct Mix8Class<(\d)> \{\s*static constexpr int kRmax = (\d+), V = (\d+), U = (\d+);"
                       r"\s*static constexpr int H\[\d+\] = \{([^}]*)\};", src)
    assert len(found) == 2
    disp = open(os.path.join(ROOT, "paper_1606_07414_gb300", "csrc", "tx16_mixed_bt.cu")).read()
    table = re.search(r"static const uint8_t H\[2\]\[8\] = \{(.*?)\};", disp, re.S).group(1)
    rows = [[int(x) for x in r.split(",")] for r in re.findall(r"\{([^{}]*)\}", table)]
    for c, rmax, V, U, H in found:
        rmax, V, U = int(rmax), int(V), int(U)
        H = [int(x) for x in H.split(",")]
        m = O.zonal_mask(rmax, 8)
        colh = [int(m[:, v].sum()) for v in range(8)]
        assert V == max(v + 1 for v in range(8) if colh[v] > 0), c
        assert U == max(colh), c
        assert H == colh[:V], c
        assert rows[int(c)] == colh, c


def test_generated_networks_are_current(tmp_path):
    """tx16_pairnet.cuh is what gen_networks.py writes today: regenerating it
    (which re-checks every emitted network against T, T^t, T8 and T8^t on
    random and unit vectors, and T8's parity and orthogonality) gives the
    committed header byte for byte."""
    import importlib.util

    csrc = os.path.join(ROOT, "paper_1606_07414_gb300", "csrc")
    spec = importlib.util.spec_from_file_location("gen_networks", os.path.join(csrc, "gen_networks.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    out = tmp_path / "pairnet.cuh"
    gen.main(str(out))
    assert out.read_bytes() == open(os.path.join(csrc, "tx16_pairnet.cuh"), "rb").read()
