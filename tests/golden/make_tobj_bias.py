"""Write ``synth/tobj_bias.json``: the objectness-logit shift of each detection anchor.

With random weights the objectness logit t_obj is centred near 0, so about half
of all anchors would pass the 0.5 confidence threshold.  This script runs the
FP64 oracle network on seeded letterboxed FullHD calibration frames at
1088x608 with no shift applied, takes the 99th percentile q of t_obj for each
(head, anchor) and stores -q, so that about 1% of anchors pass.  Only the
oracle and the input generators are used.

    python tests/golden/make_tobj_bias.py [n_frames]
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import network as net  # noqa: E402


def main(n_frames=2):
    zero = [[0.0] * 4 for _ in range(3)]
    layers = synth.parse_blob(synth.weights_blob(net.layer_specs(), tobj_shift=zero))
    t_obj = [[[] for _ in range(4)] for _ in range(3)]
    for i in range(n_frames):
        f = synth.frames_uniform(1000 + i, 1, synth.SRC_H, synth.SRC_W)
        dets, _, _ = net.forward(net.letterbox(f, 1088, 608), layers)
        for s in range(3):
            for a in range(4):
                t_obj[s][a].append(dets[s][..., 6 * a + 4].ravel())
    shift = [[-float(np.quantile(np.concatenate(t_obj[s][a]), 0.99)) for a in range(4)] for s in range(3)]
    out = dict(shift=shift, quantile=0.99, frames=n_frames, seeds=[1000 + i for i in range(n_frames)],
               input="1920x1080 uniform uint8 letterboxed to 1088x608",
               note="written by tests/golden/make_tobj_bias.py from the FP64 oracle")
    with open(os.path.join(ROOT, "synth", "tobj_bias.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 2)
