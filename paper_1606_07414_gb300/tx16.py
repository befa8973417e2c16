"""ctypes binding of libtx16 (include/tx16.h): the same entry points, with
argument marshalling from torch CUDA tensors only -- every step of the path
runs in the library's kernels.

There is no CPU fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libtx16.so")

TX16_OK, TX16_EINVAL, TX16_ENOMEM, TX16_ECUDA, TX16_ETIMEOUT, TX16_EBUSY = range(6)


class Tx16Error(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_str(status)} ({status})")
        self.status = status


class tx16_image(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("width", ctypes.c_int32), ("height", ctypes.c_int32),
                ("pitch_bytes", ctypes.c_int64), ("bits", ctypes.c_int32)]


class tx16_qparams(ctypes.Structure):
    _fields_ = [("q", ctypes.c_float), ("r", ctypes.c_int32)]


_lib = None

# name -> (restype, argtypes)
_SIGNATURES = {
    "tx16_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "tx16_image_blocks": (ctypes.c_int64, [ctypes.POINTER(tx16_image)]),
    "tx16_forward": (ctypes.c_int, [ctypes.POINTER(tx16_image), ctypes.c_int32, ctypes.c_void_p,
                                    ctypes.c_void_p]),
    "tx16_quantise": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, tx16_qparams, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    "tx16_inverse": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(tx16_image), ctypes.c_int32,
                                    ctypes.POINTER(tx16_qparams), ctypes.c_void_p]),
    "tx16_codec_batch": (ctypes.c_int, [ctypes.POINTER(tx16_image), ctypes.POINTER(tx16_image),
                                        ctypes.c_int32, ctypes.POINTER(tx16_qparams), ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p]),
    "tx16_sse": (ctypes.c_int, [ctypes.POINTER(tx16_image), ctypes.POINTER(tx16_image), ctypes.c_int32,
                                ctypes.c_void_p, ctypes.c_void_p]),
    "tx16_psnr": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(tx16_image),
                                 ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "tx16_plan_create": (ctypes.c_int, [ctypes.POINTER(tx16_image), ctypes.POINTER(tx16_image), ctypes.c_int32,
                                        ctypes.POINTER(tx16_qparams), ctypes.POINTER(ctypes.c_void_p)]),
    "tx16_plan_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tx16_plan_run_graph": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tx16_plan_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_void_p]),
    "tx16_plan_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32),
                                      ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]),
    "tx16_plan_variant": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32] + [ctypes.POINTER(ctypes.c_int32)] * 4),
    "tx16_plan_set_schedule": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int32]),
    "tx16_plan_destroy": (None, [ctypes.c_void_p]),
    "tx16_zonal_sweep": (ctypes.c_int, [ctypes.POINTER(tx16_image), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]),
    "tx16_serve_create": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_void_p)]),
    "tx16_serve_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int32, tx16_qparams, ctypes.c_void_p,
                                         ctypes.POINTER(ctypes.c_uint64)]),
    "tx16_serve_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "tx16_serve_stats": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.POINTER(ctypes.c_double)] * 4),
    "tx16_serve_reset_stats": (ctypes.c_int, [ctypes.c_void_p]),
    "tx16_serve_pause": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "tx16_serve_destroy": (None, [ctypes.c_void_p]),
    "tx16_codec_any_size": (ctypes.c_int, [ctypes.POINTER(tx16_image), ctypes.POINTER(tx16_image), ctypes.c_int32,
                                           ctypes.POINTER(tx16_qparams), ctypes.c_void_p, ctypes.c_void_p]),
    "tx16_ssim": (ctypes.c_int, [ctypes.POINTER(tx16_image), ctypes.POINTER(tx16_image), ctypes.c_int32,
                                 ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tx16_codec_mixed": (ctypes.c_int, [ctypes.POINTER(tx16_image), ctypes.POINTER(tx16_image), ctypes.c_int32,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "tx16_codec_batch_static": (ctypes.c_int, [ctypes.POINTER(tx16_image), ctypes.POINTER(tx16_image),
                                               ctypes.c_int32, ctypes.POINTER(tx16_qparams), ctypes.c_void_p,
                                               ctypes.c_void_p, ctypes.c_void_p]),
}

TX16_STATIC_MAX_IMAGES = 1024


def load(path: str | None = None) -> ctypes.CDLL:
    """Load libtx16.so (built by ``paper_1606_07414_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libtx16 is not built ({path} missing): run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def status_str(status: int) -> str:
    try:
        return load().tx16_status_str(status).decode()
    except RuntimeError:
        return f"status {status}"


def _check(status: int, what: str) -> None:
    if status != TX16_OK:
        raise Tx16Error(status, what)


# ---------------------------------------------------------------------------
# torch tensor -> descriptor marshalling
# ---------------------------------------------------------------------------
def image(t, bits: int | None = None) -> tx16_image:
    """Descriptor of a 2-D CUDA tensor of samples (uint8 for 8 bits; uint16 or
    int16 storage for 9..12 bits).  Rows may be padded (stride(0) >= width)."""
    import torch

    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("image tensors must be 2-D with unit column stride")
    esz = t.element_size()
    if bits is None:
        bits = 8 if t.dtype == torch.uint8 else 10
    if (bits == 8) != (esz == 1):
        raise ValueError("8-bit images are uint8; 9..12-bit images use 16-bit storage")
    return tx16_image(t.data_ptr(), t.shape[1], t.shape[0], t.stride(0) * esz, bits)


def _images(ts: Sequence, bits) -> ctypes.Array:
    arr = (tx16_image * max(1, len(ts)))()
    for i, t in enumerate(ts):
        arr[i] = t if isinstance(t, tx16_image) else image(t, bits)
    return arr


def _qparams(qp: Sequence[tuple[float, int]]) -> ctypes.Array:
    arr = (tx16_qparams * max(1, len(qp)))()
    for i, (q, r) in enumerate(qp):
        arr[i] = tx16_qparams(float(q) if q is not None else 0.0, int(r))
    return arr


def _stream(stream) -> ctypes.c_void_p:
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


# ---------------------------------------------------------------------------
# Entry points (names as in include/tx16.h)
# ---------------------------------------------------------------------------
def tx16_image_blocks(t, bits: int | None = None) -> int:
    d = t if isinstance(t, tx16_image) else image(t, bits)
    return int(load().tx16_image_blocks(ctypes.byref(d)))


def tx16_forward(imgs: Sequence, coeffs, stream=None, bits: int | None = None) -> None:
    """coeffs: int32 CUDA tensor with 256 * total_blocks elements."""
    lib = load()
    arr = _images(imgs, bits)
    _check(lib.tx16_forward(arr, len(imgs), _ptr(coeffs), _stream(stream)), "tx16_forward")


def tx16_quantise(coeffs, nblk: int, q: float | None, r: int, levels, stream=None) -> None:
    lib = load()
    qp = tx16_qparams(float(q) if q is not None else 0.0, int(r))
    _check(lib.tx16_quantise(_ptr(coeffs), int(nblk), qp, _ptr(levels), _stream(stream)), "tx16_quantise")


def tx16_inverse(levels, out: Sequence, qp: Sequence[tuple[float, int]], stream=None,
                 bits: int | None = None) -> None:
    lib = load()
    _check(lib.tx16_inverse(_ptr(levels), _images(out, bits), len(out), _qparams(qp), _stream(stream)),
           "tx16_inverse")


def tx16_codec_batch(inp: Sequence, out: Sequence | None, qp: Sequence[tuple[float, int]], sse=None,
                     levels=None, stream=None, bits: int | None = None) -> None:
    """Fused codec.  sse: uint64/int64 CUDA tensor of len(inp) or None."""
    lib = load()
    out_arr = _images(out, bits) if out is not None else None
    _check(lib.tx16_codec_batch(_images(inp, bits), out_arr, len(inp), _qparams(qp), _ptr(sse),
                                _ptr(levels), _stream(stream)), "tx16_codec_batch")


def tx16_codec_batch_static(inp: Sequence, out: Sequence | None, qp: Sequence[tuple[float, int]], sse=None,
                            levels=None, stream=None, bits: int | None = None) -> None:
    """tx16_codec_batch without any device allocation: for callers that cannot
    allocate device memory where they run the codec.  At most
    TX16_STATIC_MAX_IMAGES images; calls must not overlap on the GPU."""
    lib = load()
    out_arr = _images(out, bits) if out is not None else None
    _check(lib.tx16_codec_batch_static(_images(inp, bits), out_arr, len(inp), _qparams(qp), _ptr(sse),
                                       _ptr(levels), _stream(stream)), "tx16_codec_batch_static")


def tx16_zonal_sweep(imgs: Sequence, r_list: Sequence[int], sse, stream=None, bits: int | None = None) -> None:
    """sse: int64/uint64 CUDA tensor of len(imgs) * len(r_list), [image][r]."""
    lib = load()
    rl = (ctypes.c_int32 * len(r_list))(*[int(r) for r in r_list])
    _check(lib.tx16_zonal_sweep(_images(imgs, bits), len(imgs), rl, len(r_list), _ptr(sse), _stream(stream)),
           "tx16_zonal_sweep")


def tx16_codec_any_size(inp: Sequence, out: Sequence | None, qp: Sequence[tuple[float, int]], sse=None,
                        stream=None, bits: int | None = None) -> None:
    """Codec of images of any width and height (edge-replicated to whole
    blocks; only the image's own samples written and counted).  Row pitches
    must be multiples of 16 bytes: slice a wider tensor, e.g.
    ``torch.empty(h, (w + 15) // 16 * 16, dtype=torch.uint8)[:, :w]``."""
    lib = load()
    out_arr = _images(out, bits) if out is not None else None
    _check(lib.tx16_codec_any_size(_images(inp, bits), out_arr, len(inp), _qparams(qp), _ptr(sse),
                                   _stream(stream)), "tx16_codec_any_size")


def tx16_ssim(a: Sequence, b: Sequence, mssim, map=None, stream=None, bits: int | None = None) -> None:
    """Mean SSIM of each pair into ``mssim`` (float64 CUDA tensor of len(a));
    optionally every local index into ``map`` (float32 CUDA tensor holding
    sum (H - 10)(W - 10) elements, image after image)."""
    lib = load()
    _check(lib.tx16_ssim(_images(a, bits), _images(b, bits), len(a), _ptr(mssim), _ptr(map), _stream(stream)),
           "tx16_ssim")


class tx16_mixed_qparams(ctypes.Structure):
    _fields_ = [("q", ctypes.c_float), ("r16", ctypes.c_int32), ("r8", ctypes.c_int32), ("mode", ctypes.c_int32)]


MIXED_MODES = {"auto": 0, "16": 1, "8": 2}


def tx16_codec_mixed(inp: Sequence, out: Sequence | None, qp: Sequence[tuple], split=None, sse=None,
                     stream=None, bits: int | None = None) -> None:
    """Mixed 8/16 tiling.  qp: (q, r16, r8, mode) per image, mode 'auto',
    '16' or '8' (or 0, 1, 2); split: uint8 CUDA tensor, one flag per 16x16
    region, or None."""
    lib = load()
    arr = (tx16_mixed_qparams * max(1, len(qp)))()
    for i, (q, r16, r8, mode) in enumerate(qp):
        arr[i] = tx16_mixed_qparams(float(q) if q is not None else 0.0, int(r16), int(r8),
                                    MIXED_MODES.get(mode, mode) if isinstance(mode, str) else int(mode))
    out_arr = _images(out, bits) if out is not None else None
    _check(lib.tx16_codec_mixed(_images(inp, bits), out_arr, len(inp), ctypes.cast(arr, ctypes.c_void_p),
                                _ptr(split), _ptr(sse), _stream(stream)), "tx16_codec_mixed")


def tx16_sse(a: Sequence, b: Sequence, sse, stream=None, bits: int | None = None) -> None:
    lib = load()
    _check(lib.tx16_sse(_images(a, bits), _images(b, bits), len(a), _ptr(sse), _stream(stream)), "tx16_sse")


def tx16_psnr(sse_values: Sequence[int], imgs: Sequence) -> list[float]:
    """PSNR (host arithmetic in the library) from squared errors."""
    lib = load()
    n = len(sse_values)
    s = (ctypes.c_uint64 * max(1, n))(*[int(v) for v in sse_values])
    arr = (tx16_image * max(1, n))()
    for i, d in enumerate(imgs):
        arr[i] = d
    out = (ctypes.c_double * max(1, n))()
    _check(lib.tx16_psnr(s, arr, n, out), "tx16_psnr")
    return [out[i] for i in range(n)]


# ---------------------------------------------------------------------------
# Batch plans
# ---------------------------------------------------------------------------
class Plan:
    """A tx16_plan: device work list for one batch (see include/tx16.h).
    Holds references to the descriptors' tensors so they outlive the plan."""

    def __init__(self, inp: Sequence, out: Sequence | None, qp: Sequence[tuple[float, int]],
                 bits: int | None = None):
        lib = load()
        self._keep = (list(inp), list(out) if out is not None else None)
        h = ctypes.c_void_p()
        out_arr = _images(out, bits) if out is not None else None
        _check(lib.tx16_plan_create(_images(inp, bits), out_arr, len(inp), _qparams(qp), ctypes.byref(h)),
               "tx16_plan_create")
        self.handle = h
        self.n = len(inp)

    def run(self, sse=None, levels=None, stream=None) -> None:
        _check(load().tx16_plan_run(self.handle, _ptr(sse), _ptr(levels), _stream(stream)), "tx16_plan_run")

    def run_graph(self, sse=None, levels=None, stream=None) -> None:
        _check(load().tx16_plan_run_graph(self.handle, _ptr(sse), _ptr(levels), _stream(stream)),
               "tx16_plan_run_graph")

    def autotune(self, cache_path: str | None = None, stream=None) -> None:
        _check(load().tx16_plan_autotune(self.handle, cache_path.encode() if cache_path else None, _stream(stream)),
               "tx16_plan_autotune")

    def info(self) -> list[dict]:
        lib = load()
        n = ctypes.c_int32()
        m = 8
        z, t, c, k = [(ctypes.c_int32 * m)() for _ in range(4)]
        _check(lib.tx16_plan_info(self.handle, ctypes.byref(n), z, t, c, k, m), "tx16_plan_info")
        out = []
        for i in range(min(n.value, m)):
            v, w, p, s = [ctypes.c_int32() for _ in range(4)]
            _check(lib.tx16_plan_variant(self.handle, i, ctypes.byref(v), ctypes.byref(w), ctypes.byref(p),
                                         ctypes.byref(s)), "tx16_plan_variant")
            out.append({"zone": z[i], "tiles": t[i], "ctas_per_sm": c[i], "chunk": k[i], "variant": v.value,
                        "warps_per_cta": w.value, "parked_pairs": p.value, "stages": s.value})
        return out

    def set_schedule(self, run: int, variant: int, ctas_per_sm: int = 0, chunk: int = 1) -> None:
        _check(load().tx16_plan_set_schedule(self.handle, int(run), int(variant), int(ctas_per_sm), int(chunk)),
               "tx16_plan_set_schedule")

    def close(self) -> None:
        if getattr(self, "handle", None):
            load().tx16_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


def tx16_plan_create(inp: Sequence, out: Sequence | None, qp: Sequence[tuple[float, int]],
                     bits: int | None = None) -> Plan:
    return Plan(inp, out, qp, bits)


# ---------------------------------------------------------------------------
# Serving loop
# ---------------------------------------------------------------------------
class Server:
    """tx16_server: continuous-batching request loop (see include/tx16.h).
    Host buffers must be numpy arrays (pinned memory through torch is faster);
    a request's input must stay alive until its wait() returns."""

    def __init__(self, cfg: dict | None = None):
        import json

        h = ctypes.c_void_p()
        _check(load().tx16_serve_create(json.dumps(cfg).encode() if cfg else None, ctypes.byref(h)),
               "tx16_serve_create")
        self.handle = h
        self._inflight = {}

    def submit_ptr(self, in_ptr: int, w: int, h: int, bits: int, q, r: int, out_ptr: int = 0) -> int:
        t = ctypes.c_uint64()
        st = load().tx16_serve_submit(self.handle, ctypes.c_void_p(in_ptr), w, h, bits,
                                      tx16_qparams(0.0 if q is None else float(q), int(r)),
                                      ctypes.c_void_p(out_ptr), ctypes.byref(t))
        _check(st, "tx16_serve_submit")
        return t.value

    def submit(self, pixels, q, r: int, out=None, bits: int | None = None) -> int:
        """pixels/out: 2-D numpy arrays or CPU torch tensors (uint8, or uint16/int16 storage)."""
        h, w = pixels.shape[:2]
        esz = pixels.itemsize if hasattr(pixels, "itemsize") else pixels.element_size()
        bits = bits or (8 if esz == 1 else 10)
        ip = pixels.ctypes.data if hasattr(pixels, "ctypes") else pixels.data_ptr()
        op = 0 if out is None else (out.ctypes.data if hasattr(out, "ctypes") else out.data_ptr())
        t = self.submit_ptr(ip, w, h, bits, q, r, op)
        self._inflight[t] = (pixels, out)
        return t

    def wait(self, ticket: int, timeout_ms: int = 60000) -> tuple[float, float]:
        p = ctypes.c_double()
        lat = ctypes.c_double()
        st = load().tx16_serve_wait(self.handle, ticket, timeout_ms, ctypes.byref(p), ctypes.byref(lat))
        if st != TX16_ETIMEOUT:
            self._inflight.pop(ticket, None)
        _check(st, "tx16_serve_wait")
        return p.value, lat.value

    def stats(self) -> dict:
        v = [ctypes.c_double() for _ in range(4)]
        _check(load().tx16_serve_stats(self.handle, *[ctypes.byref(x) for x in v]), "tx16_serve_stats")
        return {"p50_us": v[0].value, "p99_us": v[1].value, "p999_us": v[2].value, "mblocks_per_s": v[3].value}

    def reset_stats(self) -> None:
        _check(load().tx16_serve_reset_stats(self.handle), "tx16_serve_reset_stats")

    def pause(self, paused: bool = True) -> None:
        _check(load().tx16_serve_pause(self.handle, 1 if paused else 0), "tx16_serve_pause")

    def close(self) -> None:
        if getattr(self, "handle", None):
            load().tx16_serve_destroy(self.handle)
            self.handle = None
            self._inflight.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass
