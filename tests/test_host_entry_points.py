"""Host-side logic of entry points that needs no GPU: a scene blob is checked
(format, sizes, checksum) before anything reaches the device, and the
allocation fault-injection gate is plain host state."""
import ctypes as C
import struct

import numpy as np
import pytest

from paper_2310_03505_gb300 import rr


@pytest.fixture(scope="module")
def lib():
    return rr.load()


def _fnv1a(data: bytes) -> int:
    h = 1469598103934665603
    for byte in data:
        h = ((h ^ byte) * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def _blob(payload: bytes, nv=0, nt=0, nm=1, n_tab=0, version=1, magic=b"RRSCENE\0", checksum=None,
          payload_bytes=None):
    head = struct.pack("<8s6I2Q16x", magic, version, nv, nt, nm, n_tab, 0,
                       len(payload) if payload_bytes is None else payload_bytes,
                       _fnv1a(payload) if checksum is None else checksum)
    assert len(head) == 64
    return head + payload


def _load(lib, blob: bytes):
    buf = np.frombuffer(blob, np.uint8) if blob else np.zeros(1, np.uint8)
    h = C.c_void_p()
    rc = lib.rr_scene_load(buf.ctypes.data, len(blob), C.byref(h))
    return rc, lib.rr_last_error().decode()


def _payload_bytes(nv, nt, nm, n_tab):
    mats = nm * C.sizeof(rr.rr_material)
    return nv * 12 + nt * 12 + ((nt * 2 + 3) & ~3) + mats + C.sizeof(rr.rr_batch_config) + n_tab * (4 + 4 * rr.RR_LOBE_SAMPLES)


def test_blob_layout_sizes():
    assert C.sizeof(rr.rr_material) == 24
    assert _payload_bytes(3, 1, 1, 0) == 36 + 12 + 4 + 24 + C.sizeof(rr.rr_batch_config)


@pytest.mark.parametrize("case", ["empty", "short", "magic", "version", "sizes", "checksum", "materials"])
def test_bad_blobs_are_refused_before_the_device(lib, case):
    good = bytes(_payload_bytes(0, 0, 1, 0))
    blob = {
        "empty": b"",
        "short": _blob(good)[:40],
        "magic": _blob(good, magic=b"RRSCENX\0"),
        "version": _blob(good, version=2),
        "sizes": _blob(good, payload_bytes=len(good) + 4),
        "checksum": _blob(good, checksum=_fnv1a(good) ^ 1),
        "materials": _blob(bytes(_payload_bytes(0, 0, 0, 0)), nm=0),
    }[case]
    rc, msg = _load(lib, blob)
    assert rc == rr.RR_ERR_INVALID_ARG, (case, rc, msg)


def test_fault_injection_gate_is_host_state(lib):
    seen = C.c_uint64(123)
    assert lib.rr_fault_inject_alloc(5, C.byref(seen)) == rr.RR_OK
    assert lib.rr_fault_inject_alloc(-1, C.byref(seen)) == rr.RR_OK
    assert seen.value == 0          # nothing was allocated in between
    assert lib.rr_fault_inject_alloc(-1, None) == rr.RR_OK
