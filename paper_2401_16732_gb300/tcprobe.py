"""Measured rates of the warp-level tensor-core instructions a byte-split
(digit) form of the slot contraction could be built on.  tcgen05 has no
integer kind on sm_103a, so the candidates are mma.sync u8 -> s32 and
mma.sync bf16 -> f32 with byte digits.

    python -m paper_2401_16732_gb300.tcprobe

prints one JSON line: multiply-adds/s of each, and the slot-contraction rate
each would give at best.  That best case assumes 16 digit products per
30-bit product, K = G padded to the instruction's K, and no cost for
moving operands or recombining digits.
"""
from __future__ import annotations

import json
import math

from . import flashgpu


def main():
    u8 = flashgpu.probe_mma_rate(0, 4096)
    bf = flashgpu.probe_mma_rate(1, 4096)
    out = {"mma_sync_u8_mac_per_s": u8, "mma_sync_bf16_mac_per_s": bf}
    # ResNet-18 at N=8192: G is 1, 10, 6, 4 or 3 by stage
    for name, rate, kstep in (("u8", u8, 32), ("bf16", bf, 16)):
        for G in (3, 10):
            eff = G / (kstep * math.ceil(G / kstep))
            out[f"{name}_best_slot_mac_per_s_G{G}"] = rate * eff / 16
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
