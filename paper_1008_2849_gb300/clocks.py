"""Sample the GPU's SM clock and clock-event (throttle) reasons while a timed
region runs, through NVML (libnvidia-ml, loaded with ctypes; read-only
queries only -- no clock, power or mode is ever set).  Falls back to a
polling ``nvidia-smi`` subprocess when NVML cannot be loaded.

    with ClockSampler(device_index) as cs:
        ... timed work ...
    cs.summary() -> {"sm_mhz": median, "sm_max_mhz": ..., "reasons": [...], "samples": k}
"""
from __future__ import annotations

import ctypes
import statistics
import subprocess
import threading
import time

REASONS = {
    0x1: "gpu_idle",
    0x2: "applications_clocks_setting",
    0x4: "sw_power_cap",
    0x8: "hw_slowdown",
    0x10: "sync_boost",
    0x20: "sw_thermal_slowdown",
    0x40: "hw_thermal_slowdown",
    0x80: "hw_power_brake_slowdown",
    0x100: "display_clock_setting",
}
REJECTING = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def _device_uuid(cuda_index: int):
    try:
        import torch
        u = torch.cuda.get_device_properties(cuda_index).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


class _Nvml:
    def __init__(self, cuda_index: int):
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        count = ctypes.c_uint(0)
        self.lib.nvmlDeviceGetCount_v2(ctypes.byref(count))
        want = _device_uuid(cuda_index)
        self.handle = None
        for i in range(count.value):
            h = ctypes.c_void_p()
            if self.lib.nvmlDeviceGetHandleByIndex_v2(i, ctypes.byref(h)) != 0:
                continue
            buf = ctypes.create_string_buffer(96)
            self.lib.nvmlDeviceGetUUID(h, buf, 96)
            if want is None or buf.value.decode() == want or count.value == 1:
                self.handle = h
                break
        if self.handle is None:
            raise RuntimeError("GPU not found through NVML")
        mx = ctypes.c_uint(0)
        self.lib.nvmlDeviceGetMaxClockInfo(self.handle, 1, ctypes.byref(mx))  # 1 = SM clock
        self.max_mhz = mx.value
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None)
        self.reasons_fn = fn or self.lib.nvmlDeviceGetCurrentClocksThrottleReasons

    def sample(self):
        mhz = ctypes.c_uint(0)
        self.lib.nvmlDeviceGetClockInfo(self.handle, 1, ctypes.byref(mhz))
        r = ctypes.c_ulonglong(0)
        self.reasons_fn(self.handle, ctypes.byref(r))
        return mhz.value, r.value


class ClockSampler:
    def __init__(self, cuda_index: int = 0, period_s: float = 0.002):
        self.cuda_index = cuda_index
        self.period = period_s
        self.samples = []          # (sm_mhz, reason bits)
        self.max_mhz = None
        self.source = None
        self._stop = threading.Event()
        self._thread = None
        self._proc = None

    def __enter__(self):
        try:
            self._nvml = _Nvml(self.cuda_index)
            self.max_mhz = self._nvml.max_mhz
            self.source = "nvml"
            self._thread = threading.Thread(target=self._run_nvml, daemon=True)
            self._thread.start()
        except Exception:
            self._nvml = None
            self.source = "nvidia-smi"
            self._start_smi()
        return self

    def _run_nvml(self):
        while not self._stop.is_set():
            try:
                self.samples.append(self._nvml.sample())
            except Exception:
                pass
            time.sleep(self.period)

    def _start_smi(self):
        q = "clocks.sm,clocks.max.sm,clocks_event_reasons.active"
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.cuda_index), "--query-gpu=" + q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self._proc = None

    def __exit__(self, *exc):
        self._stop.set()
        if self._thread is not None:
            self._thread.join()
            try:
                self.samples.append(self._nvml.sample())
            except Exception:
                pass
        if self._proc is not None:
            self._proc.terminate()
            out, _ = self._proc.communicate(timeout=5)
            for line in out.splitlines():
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 3:
                    try:
                        self.samples.append((int(float(parts[0])), int(parts[2], 16)))
                        self.max_mhz = int(float(parts[1]))
                    except ValueError:
                        pass
        return False

    def summary(self) -> dict:
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": [], "samples": 0,
                    "source": self.source}
        loaded = [s for s in self.samples if not (s[1] & 0x1)] or self.samples
        bits = 0
        for _, r in loaded:
            bits |= r
        reasons = [name for b, name in sorted(REASONS.items()) if bits & b and b != 0x1]
        return {"sm_mhz": statistics.median(m for m, _ in loaded), "sm_max_mhz": self.max_mhz,
                "reasons": reasons, "samples": len(loaded), "source": self.source}
