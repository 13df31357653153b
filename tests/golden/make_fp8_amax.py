"""Write fp8_amax_320x192.json: per-layer output amax of the float64 oracle forward on the seeded
calibration frames (two 1920x1080 uniform uint8 frames, seed 1000, letterboxed to 320x192).
The FP8 parity tests hand these values to the library, so both sides quantise with the same scales."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import fp8  # noqa: E402
from oracle import network as net  # noqa: E402


def main():
    layers = synth.parse_blob(synth.weights_blob(net.layer_specs()))
    x = net.letterbox(synth.frames_uniform(1000, 2, 1080, 1920), 320, 192)
    amax = fp8.calibrate(x, layers)
    out = {"what": "per-layer output amax, float64 oracle, calibration frames seed 1000 (2 frames), 320x192",
           "in": [320, 192], "amax": [float(v) for v in amax]}
    with open(os.path.join(HERE, "fp8_amax_320x192.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
