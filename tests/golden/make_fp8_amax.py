"""Write the FP8 calibration goldens: per-layer output amax of the float64 oracle forward on seeded
calibration frames (1920x1080 uniform uint8, seed 1000), letterboxed to the model input size.

* fp8_amax_320x192.json: two frames at 320x192 (the small parity configuration);
* fp8_amax_1088x608.json: one frame at 1088x608 (the batch-32 E4M3 bench configuration).

The FP8 parity tests hand these values to the library, so both sides quantise with the same scales."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import fp8  # noqa: E402
from oracle import network as net  # noqa: E402

CONFIGS = {(320, 192): 2, (1088, 608): 1}


def main(which=None):
    layers = synth.parse_blob(synth.weights_blob(net.layer_specs()))
    for (w, h), n in CONFIGS.items():
        if which and (w, h) != which:
            continue
        x = net.letterbox(synth.frames_uniform(1000, n, 1080, 1920), w, h)
        amax = fp8.calibrate(x, layers)
        out = {"what": f"per-layer output amax, float64 oracle, calibration frames seed 1000 ({n} frame"
                       f"{'s' if n > 1 else ''}), {w}x{h}",
               "in": [w, h], "amax": [float(v) for v in amax]}
        with open(os.path.join(HERE, f"fp8_amax_{w}x{h}.json"), "w") as f:
            json.dump(out, f, indent=1)


if __name__ == "__main__":
    main(tuple(int(v) for v in sys.argv[1:3]) if len(sys.argv) > 2 else None)
