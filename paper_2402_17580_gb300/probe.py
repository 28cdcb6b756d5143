"""Measure the SFU / FFMA pipe rates of the current GPU (roofline peaks).

    python -m paper_2402_17580_gb300.probe

Prints one JSON object: per op (ex2, lg2, rsqrt, rcp, ffma) the thread-level
operations per second, the SM clock the probe saw and the rate per SM per
clock.  The rcp probe alternates rcp and rsqrt (both counted); the rcp rate
alone follows from it and the rsqrt rate.
"""
import json

from ._binding import PROBE_OPS, probe_pipe


def main():
    out = {}
    for op in PROBE_OPS:
        v, mhz = probe_pipe(op)
        out[op] = {"ops_per_s": v, "sm_mhz": mhz}
    print(json.dumps(out, indent=1))
    return out


if __name__ == "__main__":
    main()
