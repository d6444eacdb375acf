"""ctypes binding of libkaze.so (the C ABI of include/kaze.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams; device images are
2-D float32 CUDA tensors with unit stride along x.  A missing library is an
error (``KazeError``), never a fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK = 0
ERR_INVALID_ARG = 1
ERR_CUDA = 2
ERR_OOM = 3
ERR_CAPACITY = 4
ERR_TIMEOUT = 5
ERR_STATE = 6

G1 = 1
G2 = 2
DOH_SIGMA4 = 0
DOH_PAPER_LITERAL = 1
SCHEME_AOS = 0
SCHEME_FED = 1
EXTREMA_3X3 = 0
EXTREMA_SIGMA_WINDOW = 1
AOS_AUTO = 0
AOS_LINES = 1
AOS_STREAMED = 2


class KazeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(msg)
        self.status = status


class Options(ctypes.Structure):
    _fields_ = [
        ("octaves", ctypes.c_int),
        ("sublevels", ctypes.c_int),
        ("sigma0", ctypes.c_float),
        ("sigma_d", ctypes.c_float),
        ("k_percentile", ctypes.c_double),
        ("nbins", ctypes.c_int),
        ("diffusivity", ctypes.c_int),
        ("dthreshold", ctypes.c_float),
        ("edge_r", ctypes.c_float),
        ("doh_norm", ctypes.c_int),
        ("k_override", ctypes.c_float),
        ("max_keypoints", ctypes.c_int),
        ("scheme", ctypes.c_int),
        ("fed_tau_max", ctypes.c_float),
        ("extrema_window", ctypes.c_int),
        ("aos_solver", ctypes.c_int),
    ]


class Keypoint(ctypes.Structure):
    _fields_ = [
        ("x", ctypes.c_float), ("y", ctypes.c_float), ("sigma", ctypes.c_float),
        ("response", ctypes.c_float), ("angle", ctypes.c_float),
        ("level", ctypes.c_int), ("octave", ctypes.c_int), ("sublevel", ctypes.c_int),
        ("ix", ctypes.c_int), ("iy", ctypes.c_int),
    ]


BATCH_PERSISTENT = 0
BATCH_CONCURRENT = 1
BATCH_RESIDENT = 2


class BatchTuning(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("cols_per_strip", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("streams", ctypes.c_int)]


KEYPOINT_DTYPE = np.dtype([
    ("x", np.float32), ("y", np.float32), ("sigma", np.float32), ("response", np.float32),
    ("angle", np.float32), ("level", np.int32), ("octave", np.int32), ("sublevel", np.int32),
    ("ix", np.int32), ("iy", np.int32),
])
assert KEYPOINT_DTYPE.itemsize == ctypes.sizeof(Keypoint) == 40

_lib = None

_vp = ctypes.c_void_p
_i = ctypes.c_int
_f = ctypes.c_float
_SIGNATURES = {
    "kaze_default_options": (None, [ctypes.POINTER(Options)]),
    "kaze_create": (_i, [ctypes.POINTER(Options), _i, _i, _vp, ctypes.POINTER(_vp)]),
    "kaze_set_stream": (_i, [_vp, _vp]),
    "kaze_build_scale_space": (_i, [_vp, _vp, _i, _i, _i]),
    "kaze_get_level": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_i), ctypes.POINTER(_f)]),
    "kaze_get_level_scale": (_i, [_vp, _i, ctypes.POINTER(_f), ctypes.POINTER(_f)]),
    "kaze_detect_enqueue": (_i, [_vp, _vp, _i, _i, _i]),
    "kaze_detect_collect": (_i, [_vp, ctypes.POINTER(Keypoint), _i, ctypes.POINTER(_i)]),
    "kaze_set_evolve_wait_limit": (_i, [_vp, ctypes.c_longlong, _i]),
    "kaze_get_contrast": (_i, [_vp, ctypes.POINTER(_f)]),
    "kaze_detector_response": (_i, [_vp]),
    "kaze_get_response": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_i)]),
    "kaze_find_extrema": (_i, [_vp, ctypes.POINTER(Keypoint), _i, ctypes.POINTER(_i)]),
    "kaze_detect": (_i, [_vp, _vp, _i, _i, _i, ctypes.POINTER(Keypoint), _i, ctypes.POINTER(_i)]),
    "kaze_detect_host": (_i, [_vp, _vp, _i, _i, _i, ctypes.POINTER(Keypoint), _i, ctypes.POINTER(_i)]),
    "kaze_detect_host_next": (_i, [_vp, _vp, _vp, _i, _i, _i, ctypes.POINTER(Keypoint), _i, ctypes.POINTER(_i)]),
    "kaze_op_gaussian": (_i, [_vp, _vp, _i, _vp, _i, _i, _i, _f]),
    "kaze_op_contrast": (_i, [_vp, _vp, _i, _i, _i, ctypes.POINTER(_f), ctypes.POINTER(_f),
                              ctypes.POINTER(ctypes.c_uint)]),
    "kaze_op_conductance": (_i, [_vp, _vp, _vp, _i, _i, _i, _f]),
    "kaze_op_aos_step": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _i, _i, _f]),
    "kaze_op_doh": (_i, [_vp, _vp, _vp, _i, _i, _i, _f, _i]),
    "kaze_op_extrema": (_i, [_vp, _vp, _i, ctypes.c_longlong, _i, _i, _i, ctypes.POINTER(_f),
                             ctypes.POINTER(Keypoint), _i, ctypes.POINTER(_i)]),
    "kaze_aos_step_static": (_i, [_vp, _vp, _vp, _i, _i, _i, _f, _vp]),
    "kaze_batch_create": (_i, [ctypes.POINTER(Options), _i, ctypes.POINTER(_i), ctypes.POINTER(_i), _vp,
                               ctypes.POINTER(_vp)]),
    "kaze_batch_detect": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_i), ctypes.POINTER(Keypoint), _i,
                               ctypes.POINTER(_i)]),
    "kaze_batch_get_level": (_i, [_vp, _i, _i, ctypes.POINTER(_vp), ctypes.POINTER(_i)]),
    "kaze_batch_get_response": (_i, [_vp, _i, _i, ctypes.POINTER(_vp), ctypes.POINTER(_i)]),
    "kaze_batch_get_tuning": (_i, [_vp, ctypes.POINTER(BatchTuning)]),
    "kaze_batch_set_tuning": (_i, [_vp, ctypes.POINTER(BatchTuning)]),
    "kaze_batch_autotune": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_i), _i, ctypes.POINTER(BatchTuning),
                                 ctypes.POINTER(ctypes.c_double)]),
    "kaze_batch_set_wait_limit": (_i, [_vp, ctypes.c_longlong, _i]),
    "kaze_batch_last_error": (ctypes.c_char_p, [_vp]),
    "kaze_batch_destroy": (None, [_vp]),
    "kaze_surrogate_create": (_i, [_i, _i, _i, _i, ctypes.c_ulonglong, _vp, ctypes.POINTER(_vp)]),
    "kaze_surrogate_set_stream": (_i, [_vp, _vp]),
    "kaze_surrogate_get_params": (_i, [_vp, ctypes.POINTER(_f), _i]),
    "kaze_surrogate_set_params": (_i, [_vp, ctypes.POINTER(_f), _i]),
    "kaze_surrogate_step": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_f),
                                 ctypes.POINTER(_vp), _i, _i, _i, _i, _i]),
    "kaze_surrogate_gradients": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_f),
                                      ctypes.POINTER(_vp), _i, _i, _i, _i, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(_f)]),
    "kaze_surrogate_train_step": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_f),
                                       ctypes.POINTER(_vp), _i, _i, _i, _i, _f, ctypes.POINTER(ctypes.c_double)]),
    "kaze_surrogate_steps_taken": (_i, [_vp, ctypes.POINTER(ctypes.c_longlong)]),
    "kaze_surrogate_sync": (_i, [_vp]),
    "kaze_surrogate_save": (_i, [_vp, ctypes.c_char_p]),
    "kaze_surrogate_load": (_i, [_vp, ctypes.c_char_p]),
    "kaze_surrogate_last_launch_count": (_i, [_vp]),
    "kaze_surrogate_last_error": (ctypes.c_char_p, [_vp]),
    "kaze_surrogate_destroy": (None, [_vp]),
    "kaze_set_surrogate": (_i, [_vp, _vp]),
    "kaze_kernel_kinds": (_i, []),
    "kaze_kernel_name": (ctypes.c_char_p, [_i]),
    "kaze_last_launch_count": (_i, [_vp]),
    "kaze_profile": (_i, [_vp, _vp, _i, _i, _i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i)]),
    "kaze_load_surrogate": (_i, [_vp, ctypes.c_char_p]),
    "kaze_build_batch": (_i, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_i), ctypes.POINTER(_i), _i, _vp, _i,
                              ctypes.POINTER(_i)]),
    "kaze_op_fed_cycle": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _i, _i, _f, ctypes.POINTER(_i)]),
    "kaze_op_fed_steps": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, ctypes.POINTER(_f), _i]),
    "kaze_describe": (_i, [_vp, _vp, _i, _vp, _i]),
    "kaze_describe_device": (_i, [_vp, _vp, _i, _vp, _i]),
    "kaze_op_describe": (_i, [_vp, _vp, _i, _i, _i, _f, _vp, _i, _vp, _i]),
    "kaze_status_string": (ctypes.c_char_p, [_i]),
    "kaze_last_error": (ctypes.c_char_p, [_vp]),
    "kaze_destroy": (None, [_vp]),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libkaze.so; raises KazeError if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise KazeError(ERR_STATE, f"libkaze.so is not built ({path}); run "
                                   "paper_1706_06750_gb300.build.build() first")
    L = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def default_options(**overrides) -> Options:
    o = Options()
    lib().kaze_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def aos_step_static(Lprev, g, Lnext, tau, stream=None):
    """One AOS step with no allocation (kaze_aos_step_static): for callers
    that cannot let the library allocate device memory.  Lprev, g, Lnext are
    2-D float32 CUDA tensors sharing one row pitch; returns the status code."""
    import torch
    w, h, pitch = _check_image(Lprev)
    for t in (g, Lnext):
        if _check_image(t) != (w, h, pitch):
            raise KazeError(ERR_INVALID_ARG, "Lprev, g and Lnext must share shape and pitch")
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(lib().kaze_aos_step_static(_vp(Lprev.data_ptr()), _vp(g.data_ptr()), _vp(Lnext.data_ptr()),
                                          pitch, w, h, float(tau), _vp(s.cuda_stream)))


class _DeviceView:
    """Zero-copy __cuda_array_interface__ over a borrowed device plane."""

    def __init__(self, ptr, h, w, pitch):
        self.__cuda_array_interface__ = {
            "shape": (h, w), "typestr": "<f4", "data": (int(ptr), False),
            "strides": (pitch * 4, 4), "version": 3,
        }


def _check_image(t):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.dim() == 2
            and t.stride(1) == 1):
        raise KazeError(ERR_INVALID_ARG, "expected a 2-D float32 CUDA tensor with unit x-stride")
    return t.shape[1], t.shape[0], t.stride(0)


def _sorted_keypoints(buf, n):
    return np.frombuffer(buf, dtype=KEYPOINT_DTYPE, count=n).copy()


class Kaze:
    """One library handle: buffers for images up to max_w x max_h."""

    def __init__(self, max_w, max_h, options: Options | None = None, stream=None, **overrides):
        import torch
        self._L = lib()
        opt = options if options is not None else default_options()
        for k, v in overrides.items():
            setattr(opt, k, v)
        self.options = opt
        if stream is None:
            # a stream of its own: the legacy default stream cannot be
            # captured into the detection graph
            stream = torch.cuda.Stream()
        self._stream = stream
        h = _vp()
        st = self._L.kaze_create(ctypes.byref(opt), int(max_w), int(max_h),
                                 _vp(stream.cuda_stream), ctypes.byref(h))
        if st != OK:
            raise KazeError(st, f"kaze_create failed: {self._L.kaze_status_string(st).decode()}: "
                                f"{self._L.kaze_last_error(None).decode()}")
        self._h = h
        self.max_w, self.max_h = int(max_w), int(max_h)
        self.n_levels = opt.octaves * opt.sublevels
        self._w = self._hh = 0
        self._kp_buf = (Keypoint * opt.max_keypoints)()

    # -- plumbing --
    def _ck(self, st, what):
        if st != OK and st != ERR_CAPACITY:
            msg = self._L.kaze_last_error(self._h).decode()
            raise KazeError(st, f"{what}: {self._L.kaze_status_string(st).decode()}: {msg}")
        return st

    def _raise_all(self, st, what):
        """Like _ck, but a capacity error raises too (nothing was done)."""
        if st == ERR_CAPACITY:
            msg = self._L.kaze_last_error(self._h).decode()
            raise KazeError(st, f"{what}: {self._L.kaze_status_string(st).decode()}: {msg}")
        return self._ck(st, what)

    def close(self):
        if getattr(self, "_h", None):
            self._L.kaze_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h.value

    @property
    def stream(self):
        """The torch.cuda.Stream the handle enqueues on."""
        return self._stream

    def _begin(self):
        # order the handle's stream after work already queued by the caller
        import torch
        cur = torch.cuda.current_stream()
        if cur != self._stream:
            self._stream.wait_stream(cur)

    def _end(self):
        # and the caller's stream after the handle's work
        import torch
        cur = torch.cuda.current_stream()
        if cur != self._stream:
            cur.wait_stream(self._stream)

    # -- pipeline --
    def build_scale_space(self, img):
        w, h, pitch = _check_image(img)
        self._begin()
        self._ck(self._L.kaze_build_scale_space(self._h, _vp(img.data_ptr()), w, h, pitch),
                 "kaze_build_scale_space")
        self._end()
        self._w, self._hh = w, h

    def level(self, i, copy=True):
        import torch
        p = _vp()
        pitch = _i()
        t = _f()
        self._ck(self._L.kaze_get_level(self._h, int(i), ctypes.byref(p), ctypes.byref(pitch),
                                        ctypes.byref(t)), "kaze_get_level")
        v = torch.as_tensor(_DeviceView(p.value, self._hh, self._w, pitch.value), device="cuda")
        return v.clone() if copy else v

    def levels(self):
        import torch
        return torch.stack([self.level(i) for i in range(self.n_levels)])

    def level_sigma(self, i):
        """sigma_i of level i as the library holds it (Eq. 6, FP32)."""
        s = _f()
        self._ck(self._L.kaze_get_level_scale(self._h, int(i), ctypes.byref(s), None), "kaze_get_level_scale")
        return float(s.value)

    def set_evolve_wait_limit(self, cycles, stall_tile=-1):
        """Failure-detection hook of the resident evolution: a grid-barrier
        wait gives up after `cycles`; stall_tile >= 0 makes that tile never
        arrive (kaze_set_evolve_wait_limit)."""
        self._ck(self._L.kaze_set_evolve_wait_limit(self._h, int(cycles), int(stall_tile)),
                 "kaze_set_evolve_wait_limit")

    def level_time(self, i):
        t = _f()
        self._ck(self._L.kaze_get_level(self._h, int(i), None, None, ctypes.byref(t)), "kaze_get_level")
        return float(t.value)

    def contrast(self):
        k = _f()
        self._ck(self._L.kaze_get_contrast(self._h, ctypes.byref(k)), "kaze_get_contrast")
        return float(k.value)

    def detector_response(self):
        self._begin()
        self._ck(self._L.kaze_detector_response(self._h), "kaze_detector_response")
        self._end()

    def response(self, i, copy=True):
        import torch
        p = _vp()
        pitch = _i()
        self._ck(self._L.kaze_get_response(self._h, int(i), ctypes.byref(p), ctypes.byref(pitch)),
                 "kaze_get_response")
        v = torch.as_tensor(_DeviceView(p.value, self._hh, self._w, pitch.value), device="cuda")
        return v.clone() if copy else v

    def responses(self):
        import torch
        return torch.stack([self.response(i) for i in range(self.n_levels)])

    def find_extrema(self, capacity=None):
        """Keypoints sorted by (level, iy, ix) as a KEYPOINT_DTYPE array."""
        cap = self.options.max_keypoints if capacity is None else int(capacity)
        buf = self._kp_buf if cap <= len(self._kp_buf) else (Keypoint * cap)()
        n = _i()
        self._begin()
        st = self._ck(self._L.kaze_find_extrema(self._h, buf, cap, ctypes.byref(n)), "kaze_find_extrema")
        self._end()
        self.last_status = st
        self.last_count = n.value
        return _sorted_keypoints(buf, min(n.value, cap))

    def detect(self, img, capacity=None):
        """Scale space + response + extrema of a device image (graph-replayed)."""
        w, h, pitch = _check_image(img)
        cap = self.options.max_keypoints if capacity is None else int(capacity)
        buf = self._kp_buf if cap <= len(self._kp_buf) else (Keypoint * cap)()
        n = _i()
        self._begin()
        st = self._ck(self._L.kaze_detect(self._h, _vp(img.data_ptr()), w, h, pitch, buf, cap,
                                          ctypes.byref(n)), "kaze_detect")
        self._end()
        self._w, self._hh = w, h
        self.last_status = st
        self.last_count = n.value
        return _sorted_keypoints(buf, min(n.value, cap))

    def detect_enqueue(self, img):
        """The first half of detect: replay the detection without waiting."""
        w, h, pitch = _check_image(img)
        self._begin()
        self._ck(self._L.kaze_detect_enqueue(self._h, _vp(img.data_ptr()), w, h, pitch), "kaze_detect_enqueue")
        self._w, self._hh = w, h

    def detect_collect(self, capacity=None):
        """The second half of detect: wait for the enqueued detection and
        return its keypoints."""
        cap = self.options.max_keypoints if capacity is None else int(capacity)
        buf = self._kp_buf if cap <= len(self._kp_buf) else (Keypoint * cap)()
        n = _i()
        self._begin()
        st = self._ck(self._L.kaze_detect_collect(self._h, buf, cap, ctypes.byref(n)), "kaze_detect_collect")
        self._end()
        self.last_status = st
        self.last_count = n.value
        return _sorted_keypoints(buf, min(n.value, cap))

    @staticmethod
    def _host_image(img):
        """(pointer, h, w, pitch, keep-alive) of a 2-D float32 host image."""
        import torch
        if isinstance(img, torch.Tensor):
            if img.is_cuda or img.dtype != torch.float32 or img.dim() != 2 or img.stride(1) != 1:
                raise KazeError(ERR_INVALID_ARG, "expected a 2-D float32 CPU tensor")
            return img.data_ptr(), img.shape[0], img.shape[1], img.stride(0), img
        img = np.ascontiguousarray(img, dtype=np.float32)
        return img.ctypes.data, img.shape[0], img.shape[1], img.shape[1], img

    def detect_host(self, img, capacity=None, next_image=None):
        """kaze_detect on a host image (numpy array or CPU tensor, float32).
        With `next_image` (the following image: same size and row stride, kept
        alive and unchanged until it is detected, ideally pinned), its copy to
        the device starts while `img` is detected (kaze_detect_host_next)."""
        ptr, h, w, pitch, keep = self._host_image(img)
        if next_image is not None:
            nptr, nh, nw, npitch, nkeep = self._host_image(next_image)
            if (nh, nw, npitch) != (h, w, pitch):
                raise KazeError(ERR_INVALID_ARG, "the next image must have the same size and row stride")
        cap = self.options.max_keypoints if capacity is None else int(capacity)
        buf = self._kp_buf if cap <= len(self._kp_buf) else (Keypoint * cap)()
        n = _i()
        self._begin()
        if next_image is None:
            st = self._ck(self._L.kaze_detect_host(self._h, _vp(ptr), w, h, pitch, buf, cap, ctypes.byref(n)),
                          "kaze_detect_host")
        else:
            self._next_keep = nkeep  # the copy reads it after this call returns
            st = self._ck(self._L.kaze_detect_host_next(self._h, _vp(ptr), _vp(nptr), w, h, pitch, buf, cap,
                                                        ctypes.byref(n)), "kaze_detect_host_next")
        del keep
        self._end()
        self._w, self._hh = w, h
        self.last_status = st
        self.last_count = n.value
        return _sorted_keypoints(buf, min(n.value, cap))

    # -- description (Sec. II-C) --
    def describe(self, keypoints, upright=False):
        """Orientation and 64-D M-SURF descriptor of keypoints (a KEYPOINT_DTYPE
        array, e.g. from detect) on the levels of the last build.  Returns a
        copy of the keypoints with their angle set and the [n, 64] float32
        descriptors."""
        kp = np.ascontiguousarray(np.asarray(keypoints, dtype=KEYPOINT_DTYPE)).copy()
        n = len(kp)
        desc = np.zeros((n, 64), dtype=np.float32)
        self._begin()
        st = self._L.kaze_describe(self._h, _vp(kp.ctypes.data if n else None), n,
                                   _vp(desc.ctypes.data if n else None), int(bool(upright)))
        self._end()
        self._raise_all(st, "kaze_describe")
        return kp, desc

    def describe_device(self, d_kps, d_desc, n, upright=False):
        """kaze_describe_device on device buffers: d_kps a CUDA tensor holding
        n keypoint records (see keypoints_to_device), d_desc a [n, 64] float32
        CUDA tensor.  Asynchronous on the handle's stream."""
        self._begin()
        self._ck(self._L.kaze_describe_device(self._h, _vp(d_kps.data_ptr()), int(n), _vp(d_desc.data_ptr()),
                                              int(bool(upright))), "kaze_describe_device")
        self._end()

    @staticmethod
    def keypoints_to_device(keypoints):
        """A CUDA uint8 tensor holding the keypoint records byte for byte."""
        import torch
        kp = np.ascontiguousarray(np.asarray(keypoints, dtype=KEYPOINT_DTYPE))
        return torch.from_numpy(kp.view(np.uint8).copy()).cuda()

    @staticmethod
    def keypoints_from_device(t, n):
        return np.frombuffer(t[: n * KEYPOINT_DTYPE.itemsize].cpu().numpy().tobytes(), dtype=KEYPOINT_DTYPE,
                             count=n).copy()

    def op_describe(self, L, sigma, points, upright=False):
        """Description on one given level image L (2-D float32 CUDA tensor) of
        scale sigma at points: a KEYPOINT_DTYPE array or a sequence of (x, y).
        Returns (angles [n], descriptors [n, 64])."""
        w, h, pitch = _check_image(L)
        if isinstance(points, np.ndarray) and points.dtype == KEYPOINT_DTYPE:
            kp = np.ascontiguousarray(points).copy()
        else:
            pts = list(points)
            kp = np.zeros(len(pts), dtype=KEYPOINT_DTYPE)
            for i, (x, y) in enumerate(pts):
                kp[i]["x"], kp[i]["y"] = x, y
        n = len(kp)
        desc = np.zeros((n, 64), dtype=np.float32)
        self._begin()
        st = self._L.kaze_op_describe(self._h, _vp(L.data_ptr()), pitch, w, h, float(sigma),
                                      _vp(kp.ctypes.data if n else None), n,
                                      _vp(desc.ctypes.data if n else None), int(bool(upright)))
        self._end()
        self._raise_all(st, "kaze_op_describe")
        return kp["angle"].astype(np.float64), desc

    # -- instrumentation --
    def set_surrogate(self, surrogate):
        """Evolve the scale space with the learned surrogate's fused step
        instead of AOS (None restores AOS).  The Surrogate must outlive its
        use here."""
        self._ck(self._L.kaze_set_surrogate(self._h, surrogate._s if surrogate is not None else None),
                 "kaze_set_surrogate")
        self._surrogate = surrogate

    def load_surrogate(self, path):
        """Evolve with a surrogate checkpoint the handle loads and owns
        (None restores AOS)."""
        self._ck(self._L.kaze_load_surrogate(self._h, None if path is None else os.fsencode(path)),
                 "kaze_load_surrogate")

    def build_batch(self, imgs, capacity=None):
        """Detection of a list of 2-D float32 CUDA tensors (contiguous rows)
        through one batch with the handle's options; a list of keypoint
        arrays, one per image."""
        n = len(imgs)
        for t in imgs:
            w, h, pitch = _check_image(t)
            if pitch != w:
                raise KazeError(ERR_INVALID_ARG, "build_batch needs contiguous rows (pitch == width)")
        ptrs = (_vp * n)(*[t.data_ptr() for t in imgs])
        ws = (_i * n)(*[t.shape[1] for t in imgs])
        hs = (_i * n)(*[t.shape[0] for t in imgs])
        cap = self.options.max_keypoints if capacity is None else int(capacity)
        buf = (Keypoint * (cap * n))()
        counts = (_i * n)()
        self._begin()
        st = self._ck(self._L.kaze_build_batch(self._h, ptrs, ws, hs, n, buf, cap, counts), "kaze_build_batch")
        self._end()
        self.last_status = st
        raw = np.frombuffer(buf, dtype=KEYPOINT_DTYPE, count=cap * n)
        return [raw[i * cap: i * cap + min(counts[i], cap)].copy() for i in range(n)]

    def last_launch_count(self):
        return int(self._L.kaze_last_launch_count(self._h))

    def profile(self, img):
        """One eager pipeline pass with per-kernel CUDA events.

        Returns {kernel kind: (summed ms, launches)}."""
        w, h, pitch = _check_image(img)
        nk = self._L.kaze_kernel_kinds()
        ms = (ctypes.c_double * nk)()
        cnt = (_i * nk)()
        self._begin()
        self._ck(self._L.kaze_profile(self._h, _vp(img.data_ptr()), w, h, pitch, ms, cnt), "kaze_profile")
        self._end()
        self._w, self._hh = w, h
        return {self._L.kaze_kernel_name(k).decode(): (float(ms[k]), int(cnt[k])) for k in range(nk)}

    # -- single steps --
    def op_gaussian(self, src, dst, sigma):
        w, h, pin = _check_image(src)
        _, _, pout = _check_image(dst)
        self._begin()
        self._ck(self._L.kaze_op_gaussian(self._h, _vp(src.data_ptr()), pin, _vp(dst.data_ptr()), pout,
                                          w, h, float(sigma)), "kaze_op_gaussian")
        self._end()

    def op_contrast(self, L0):
        w, h, pitch = _check_image(L0)
        k = _f()
        hm = _f()
        hist = (ctypes.c_uint * self.options.nbins)()
        self._begin()
        self._ck(self._L.kaze_op_contrast(self._h, _vp(L0.data_ptr()), pitch, w, h, ctypes.byref(k),
                                          ctypes.byref(hm), hist), "kaze_op_contrast")
        self._end()
        return float(k.value), float(hm.value), np.array(hist, dtype=np.int64)

    def op_conductance(self, L, g, k):
        w, h, pitch = _check_image(L)
        self._begin()
        self._ck(self._L.kaze_op_conductance(self._h, _vp(L.data_ptr()), _vp(g.data_ptr()), pitch, w, h,
                                             float(k)), "kaze_op_conductance")
        self._end()

    def op_aos_step(self, Lprev, g, ux, Lnext, tau):
        w, h, pitch = _check_image(Lprev)
        self._begin()
        self._ck(self._L.kaze_op_aos_step(self._h, _vp(Lprev.data_ptr()), _vp(g.data_ptr()),
                                          _vp(ux.data_ptr()), _vp(Lnext.data_ptr()), pitch, w, h,
                                          float(tau)), "kaze_op_aos_step")
        self._end()

    def op_fed_cycle(self, Lprev, g, scratch, Lnext, dt):
        """One FED cycle (Eq. 5) from Lprev to stopping time dt with g fixed;
        returns the number of explicit steps."""
        w, h, pitch = _check_image(Lprev)
        n = _i()
        self._begin()
        self._ck(self._L.kaze_op_fed_cycle(self._h, _vp(Lprev.data_ptr()), _vp(g.data_ptr()),
                                           _vp(scratch.data_ptr()), _vp(Lnext.data_ptr()), pitch, w, h,
                                           float(dt), ctypes.byref(n)), "kaze_op_fed_cycle")
        self._end()
        return int(n.value)

    def op_fed_steps(self, Lprev, g, Lnext, taus):
        """len(taus) (1..4) explicit steps of Eq. 5 from Lprev into Lnext in
        one launch, g fixed."""
        w, h, pitch = _check_image(Lprev)
        t = (_f * max(len(taus), 1))(*[float(v) for v in taus])
        self._begin()
        self._ck(self._L.kaze_op_fed_steps(self._h, _vp(Lprev.data_ptr()), _vp(g.data_ptr()),
                                           _vp(Lnext.data_ptr()), pitch, w, h, t, len(taus)),
                 "kaze_op_fed_steps")
        self._end()

    def op_doh(self, L, D, sigma_i, octave):
        w, h, pitch = _check_image(L)
        self._begin()
        self._ck(self._L.kaze_op_doh(self._h, _vp(L.data_ptr()), _vp(D.data_ptr()), pitch, w, h,
                                     float(sigma_i), int(octave)), "kaze_op_doh")
        self._end()

    def op_extrema(self, D, sigma, capacity=None):
        """D: [n, h, w] float32 CUDA tensor (contiguous rows)."""
        import torch
        if not (isinstance(D, torch.Tensor) and D.is_cuda and D.dim() == 3 and D.stride(2) == 1
                and D.dtype == torch.float32):
            raise KazeError(ERR_INVALID_ARG, "expected a [n, h, w] float32 CUDA tensor")
        n, h, w = D.shape
        sig = (ctypes.c_float * n)(*[float(s) for s in sigma])
        cap = self.options.max_keypoints if capacity is None else int(capacity)
        buf = self._kp_buf if cap <= len(self._kp_buf) else (Keypoint * cap)()
        cnt = _i()
        self._begin()
        st = self._ck(self._L.kaze_op_extrema(self._h, _vp(D.data_ptr()), D.stride(1), D.stride(0), w, h, n,
                                              sig, buf, cap, ctypes.byref(cnt)), "kaze_op_extrema")
        self._end()
        self.last_status = st
        self.last_count = cnt.value
        return _sorted_keypoints(buf, min(cnt.value, cap))


class Batch:
    """A batch handle (kaze_batch): the whole detection of a fixed list of
    images of mixed sizes in one persistent launch."""

    def __init__(self, sizes, options: Options | None = None, stream=None, **overrides):
        import torch
        self._L = lib()
        opt = options if options is not None else default_options()
        for k, v in overrides.items():
            setattr(opt, k, v)
        self.options = opt
        self.sizes = [(int(w), int(h)) for w, h in sizes]
        self.n = len(self.sizes)
        self.n_levels = opt.octaves * opt.sublevels
        self._stream = stream if stream is not None else torch.cuda.Stream()
        ws = (_i * self.n)(*[w for w, _ in self.sizes])
        hs = (_i * self.n)(*[h for _, h in self.sizes])
        h = _vp()
        st = self._L.kaze_batch_create(ctypes.byref(opt), self.n, ws, hs, _vp(self._stream.cuda_stream),
                                       ctypes.byref(h))
        if st != OK:
            raise KazeError(st, f"kaze_batch_create failed: {self._L.kaze_status_string(st).decode()}")
        self._h = h
        self._cap = opt.max_keypoints
        self._kp_buf = None

    def _ck(self, st, what):
        if st != OK and st != ERR_CAPACITY:
            msg = self._L.kaze_batch_last_error(self._h).decode()
            raise KazeError(st, f"{what}: {self._L.kaze_status_string(st).decode()}: {msg}")
        return st

    def close(self):
        if getattr(self, "_h", None):
            self._L.kaze_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def stream(self):
        return self._stream

    def _inputs(self, imgs):
        if len(imgs) != self.n:
            raise KazeError(ERR_INVALID_ARG, f"expected {self.n} images")
        ptrs = (_vp * self.n)()
        pitches = (_i * self.n)()
        for i, t in enumerate(imgs):
            w, h, pitch = _check_image(t)
            if (w, h) != self.sizes[i]:
                raise KazeError(ERR_INVALID_ARG, f"image {i} is {w}x{h}, expected {self.sizes[i]}")
            ptrs[i] = t.data_ptr()
            pitches[i] = pitch
        return ptrs, pitches

    def _begin(self):
        import torch
        cur = torch.cuda.current_stream()
        if cur != self._stream:
            self._stream.wait_stream(cur)

    def detect(self, imgs, capacity=None):
        """Keypoints of every image: a list of KEYPOINT_DTYPE arrays."""
        cap = self._cap if capacity is None else int(capacity)
        ptrs, pitches = self._inputs(imgs)
        if self._kp_buf is None or len(self._kp_buf) < cap * self.n:
            self._kp_buf = (Keypoint * (cap * self.n))()
        counts = (_i * self.n)()
        self._begin()
        st = self._ck(self._L.kaze_batch_detect(self._h, ptrs, pitches, self._kp_buf, cap, counts),
                      "kaze_batch_detect")
        self.last_status = st
        self.last_counts = list(counts)
        raw = np.frombuffer(self._kp_buf, dtype=KEYPOINT_DTYPE, count=cap * self.n)
        return [raw[i * cap: i * cap + min(counts[i], cap)].copy() for i in range(self.n)]

    def level(self, image, level):
        import torch
        p = _vp()
        pitch = _i()
        self._ck(self._L.kaze_batch_get_level(self._h, int(image), int(level), ctypes.byref(p),
                                              ctypes.byref(pitch)), "kaze_batch_get_level")
        w, h = self.sizes[image]
        return torch.as_tensor(_DeviceView(p.value, h, w, pitch.value), device="cuda").clone()

    def response(self, image, level):
        import torch
        p = _vp()
        pitch = _i()
        self._ck(self._L.kaze_batch_get_response(self._h, int(image), int(level), ctypes.byref(p),
                                                 ctypes.byref(pitch)), "kaze_batch_get_response")
        w, h = self.sizes[image]
        return torch.as_tensor(_DeviceView(p.value, h, w, pitch.value), device="cuda").clone()

    def tuning(self):
        """(mode, cols_per_strip, ctas_per_sm, streams)"""
        t = BatchTuning()
        self._ck(self._L.kaze_batch_get_tuning(self._h, ctypes.byref(t)), "kaze_batch_get_tuning")
        return (t.mode, t.cols_per_strip, t.ctas_per_sm, t.streams)

    def set_tuning(self, mode=BATCH_PERSISTENT, cols_per_strip=4, ctas_per_sm=2, streams=8):
        t = BatchTuning(int(mode), int(cols_per_strip), int(ctas_per_sm), int(streams))
        self._ck(self._L.kaze_batch_set_tuning(self._h, ctypes.byref(t)), "kaze_batch_set_tuning")

    def autotune(self, imgs, reps=3, cache=None):
        """Times every solve-tile shape on these images and keeps the fastest.

        With `cache` (a JSON path) the choice is stored under a key made of
        the device name and the size list, and reused when present."""
        import json
        import os
        import torch
        key = None
        if cache:
            key = torch.cuda.get_device_name() + "|" + ",".join(f"{w}x{h}" for w, h in sorted(self.sizes))
            try:
                with open(cache) as f:
                    known = json.load(f)
                if key in known:
                    self.set_tuning(*known[key]["tuning"])
                    return tuple(known[key]["tuning"]), known[key]["ms"]
            except (OSError, ValueError, KeyError):
                pass
        ptrs, pitches = self._inputs(imgs)
        best = BatchTuning()
        ms = ctypes.c_double()
        self._begin()
        self._ck(self._L.kaze_batch_autotune(self._h, ptrs, pitches, int(reps), ctypes.byref(best),
                                             ctypes.byref(ms)), "kaze_batch_autotune")
        result = (best.mode, best.cols_per_strip, best.ctas_per_sm, best.streams)
        if cache:
            try:
                with open(cache) as f:
                    known = json.load(f)
            except (OSError, ValueError):
                known = {}
            known[key] = {"tuning": list(result), "ms": ms.value}
            os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
            with open(cache, "w") as f:
                json.dump(known, f, indent=1)
        return result, ms.value

    def set_wait_limit(self, cycles, stall_image=-1):
        """Test hook: bound of a device-side wait in SM cycles; stall_image
        >= 0 makes one stage of that image wait for an item that never
        exists, so the next detect reports ERR_TIMEOUT."""
        self._ck(self._L.kaze_batch_set_wait_limit(self._h, int(cycles), int(stall_image)),
                 "kaze_batch_set_wait_limit")


SURROGATE_PARAMS = 20257
SURROGATE_MAX_SAMPLES = 64
SURROGATE_TRAIN = 1
SURROGATE_FUSED = 0
SURROGATE_LAYERED = 1
SURROGATE_FUSED_SYNC = 2


def _planes(x, name):
    """A list of 2-D float32 CUDA tensors (or one 3-D tensor [n, h, w]) ->
    (n, w, h, pitch, ctypes array of device pointers).  Every plane must
    share shape and row pitch."""
    import torch
    if isinstance(x, torch.Tensor) and x.dim() == 3:
        x = [x[i] for i in range(x.shape[0])]
    elif isinstance(x, torch.Tensor):
        x = [x]
    if not x:
        raise KazeError(ERR_INVALID_ARG, f"{name}: no planes")
    geo = None
    for t in x:
        g = _check_image(t)
        if geo is not None and g != geo:
            raise KazeError(ERR_INVALID_ARG, f"{name}: planes differ in shape or pitch")
        geo = g
    arr = (_vp * len(x))(*[t.data_ptr() for t in x])
    return len(x), geo[0], geo[1], geo[2], arr


class Surrogate:
    """The learned stand-in for one AOS step (kaze_surrogate_*): a 4-layer
    3x3 convolutional network, BF16 weights, FP32 accumulation."""

    def __init__(self, max_w=0, max_h=0, max_samples=0, train=False, seed=0, stream=None):
        import torch
        self._L = lib()
        if stream is None:
            stream = torch.cuda.Stream()
        self._stream = stream
        s = _vp()
        st = self._L.kaze_surrogate_create(int(max_w), int(max_h), int(max_samples),
                                           SURROGATE_TRAIN if train else 0, int(seed),
                                           _vp(stream.cuda_stream), ctypes.byref(s))
        if st != OK:
            raise KazeError(st, f"kaze_surrogate_create failed: {self._L.kaze_status_string(st).decode()}: "
                                f"{self._L.kaze_surrogate_last_error(None).decode()}")
        self._s = s

    def _ck(self, st, what):
        if st != OK:
            msg = self._L.kaze_surrogate_last_error(self._s).decode()
            raise KazeError(st, f"{what}: {self._L.kaze_status_string(st).decode()}: {msg}")
        return st

    def close(self):
        if getattr(self, "_s", None):
            self._L.kaze_surrogate_destroy(self._s)
            self._s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def stream(self):
        return self._stream

    def _begin(self):
        import torch
        cur = torch.cuda.current_stream()
        if cur != self._stream:
            self._stream.wait_stream(cur)

    def _end(self):
        import torch
        cur = torch.cuda.current_stream()
        if cur != self._stream:
            cur.wait_stream(self._stream)

    def _batch(self, L, g, tau, T=None):
        n, w, h, pitch, pl = _planes(L, "L")
        ng, wg, hg, pg, pg_arr = _planes(g, "g")
        if (ng, wg, hg, pg) != (n, w, h, pitch):
            raise KazeError(ERR_INVALID_ARG, "g must match L")
        taus = np.broadcast_to(np.asarray(tau, dtype=np.float32), (n,)).copy()
        ta = taus.ctypes.data_as(ctypes.POINTER(_f))
        pt = None
        if T is not None:
            nt, wt, ht, ptc, pt = _planes(T, "T")
            if (nt, wt, ht, ptc) != (n, w, h, pitch):
                raise KazeError(ERR_INVALID_ARG, "T must match L")
        return n, w, h, pitch, pl, pg_arr, taus, ta, pt

    def step(self, L, g, tau, out, path=SURROGATE_FUSED):
        """out[i] = L_next of (L[i], g[i], tau[i]); asynchronous."""
        n, w, h, pitch, pl, pg, taus, ta, _ = self._batch(L, g, tau)
        no, wo, ho, po, pout = _planes(out, "out")
        if (no, wo, ho, po) != (n, w, h, pitch):
            raise KazeError(ERR_INVALID_ARG, "out must match L")
        self._begin()
        self._ck(self._L.kaze_surrogate_step(self._s, pl, pg, ta, pout, n, w, h, pitch, int(path)),
                 "kaze_surrogate_step")
        self._end()

    def gradients(self, L, g, tau, T):
        """(loss, gradient) of the mean squared error against T."""
        n, w, h, pitch, pl, pg, taus, ta, pt = self._batch(L, g, tau, T)
        grad = np.zeros(SURROGATE_PARAMS, dtype=np.float32)
        loss = ctypes.c_double(0.0)
        self._begin()
        self._ck(self._L.kaze_surrogate_gradients(self._s, pl, pg, ta, pt, n, w, h, pitch, ctypes.byref(loss),
                                                  grad.ctypes.data_as(ctypes.POINTER(_f))),
                 "kaze_surrogate_gradients")
        self._end()
        return float(loss.value), grad

    def train_step(self, L, g, tau, T, lr, want_loss=True):
        """One Adam step; returns the loss before it (None if not wanted)."""
        n, w, h, pitch, pl, pg, taus, ta, pt = self._batch(L, g, tau, T)
        loss = ctypes.c_double(0.0)
        self._begin()
        self._ck(self._L.kaze_surrogate_train_step(self._s, pl, pg, ta, pt, n, w, h, pitch, float(lr),
                                                   ctypes.byref(loss) if want_loss else None),
                 "kaze_surrogate_train_step")
        self._end()
        return float(loss.value) if want_loss else None

    def params(self):
        p = np.zeros(SURROGATE_PARAMS, dtype=np.float32)
        self._ck(self._L.kaze_surrogate_get_params(self._s, p.ctypes.data_as(ctypes.POINTER(_f)), p.size),
                 "kaze_surrogate_get_params")
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.shape != (SURROGATE_PARAMS,):
            raise KazeError(ERR_INVALID_ARG, f"expected {SURROGATE_PARAMS} parameters")
        self._ck(self._L.kaze_surrogate_set_params(self._s, p.ctypes.data_as(ctypes.POINTER(_f)), p.size),
                 "kaze_surrogate_set_params")

    def sync(self):
        """Waits for the surrogate's stream; raises on a device-side timeout."""
        self._ck(self._L.kaze_surrogate_sync(self._s), "kaze_surrogate_sync")

    def steps_taken(self):
        n = ctypes.c_longlong(0)
        self._ck(self._L.kaze_surrogate_steps_taken(self._s, ctypes.byref(n)), "kaze_surrogate_steps_taken")
        return int(n.value)

    def save(self, path):
        self._ck(self._L.kaze_surrogate_save(self._s, os.fsencode(path)), "kaze_surrogate_save")

    def load(self, path):
        self._ck(self._L.kaze_surrogate_load(self._s, os.fsencode(path)), "kaze_surrogate_load")

    def last_launch_count(self):
        return int(self._L.kaze_surrogate_last_launch_count(self._s))
