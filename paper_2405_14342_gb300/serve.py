"""Python front end of the librogs serving loop (rogs_serve_*).

The loop itself -- admission by free device memory, continuous batching of
requests into one forward pass, overlap of batches on several streams,
packing of the RGB / semantic / elevation channels -- runs inside the C
library; this class only marshals cameras and decodes the packed results.
"""
from __future__ import annotations

import ctypes as C
import time

import numpy as np

from . import rogs as R

RGB, SEM, ELEV = R.ROGS_CH_RGB, R.ROGS_CH_SEM, R.ROGS_CH_ELEV


class Server:
    def __init__(self, renderer_cfg: R.rogs_config, surfels, exposure, max_batch_views=16, max_inflight=3,
                 max_queue=4096, memory_budget=8 << 30, record_capacity=4_000_000, pair_capacity=24_000_000,
                 timeout_s=30.0):
        cfg = R.rogs_serve_config(max_batch_views=max_batch_views, max_inflight=max_inflight, max_queue=max_queue,
                                  reserved=0, memory_budget=int(memory_budget), record_capacity=int(record_capacity),
                                  pair_capacity=int(pair_capacity), timeout_s=float(timeout_s))
        self.C = int(renderer_cfg.num_classes)
        self._surf = surfels                      # keep the device tensors alive
        self._exposure = exposure
        self.h = R.rogs_serve_open(renderer_cfg, surfels.c_struct(), exposure, cfg)
        self._meta = {}

    def submit(self, cam, channels=RGB) -> int:
        arr = R.cameras([cam])
        t = R.rogs_serve_submit(self.h, arr, channels)
        nbytes = R.rogs_serve_result_bytes(arr, channels, self.C)
        self._meta[t] = (cam.width, cam.height, channels, nbytes)
        return t

    def poll(self, ticket):
        """None while pending, else a dict of numpy arrays (rgb [3,H,W], elev [H,W], sem [H,W] uint8)."""
        W, H, ch, nbytes = self._meta[ticket]
        buf = np.empty(max(nbytes, 1), np.uint8)
        if not R.rogs_serve_poll(self.h, ticket, buf.ctypes.data_as(C.c_void_p)):
            return None
        del self._meta[ticket]
        return decode(buf, W, H, ch)

    def wait(self, ticket, timeout=60.0, sleep=5e-5):
        t0 = time.perf_counter()
        while True:
            r = self.poll(ticket)
            if r is not None:
                return r
            if time.perf_counter() - t0 > timeout:
                raise TimeoutError(f"request {ticket} not finished after {timeout} s")
            time.sleep(sleep)

    def set_timeout(self, timeout_s: float):
        R.rogs_serve_set_timeout(self.h, timeout_s)

    def stats(self) -> R.rogs_serve_stats:
        return R.rogs_serve_get_stats(self.h)

    def close(self):
        if self.h:
            R.rogs_serve_close(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def decode(buf: np.ndarray, W: int, H: int, channels: int) -> dict:
    P = W * H
    out, off = {}, 0
    if channels & RGB:
        out["rgb"] = buf[off: off + 12 * P].view(np.float32).reshape(3, H, W)
        off += 12 * P
    if channels & ELEV:
        out["elev"] = buf[off: off + 4 * P].view(np.float32).reshape(H, W)
        off += 4 * P
    if channels & SEM:
        out["sem"] = buf[off: off + P].reshape(H, W)
        off += P
    return out
