"""Device decode of Motion-JPEG frames (jde_decode_jpeg): decoded frames against their source, the
host-side header check, and the decoded frames through the detector."""
import numpy as np
import pytest
import torch

import synth
from gpu_helpers import jde

pytestmark = pytest.mark.gpu


def _decoder(j, n=4):
    try:
        return j.jde_decoder_create(0, n, True)
    except j.JdeError as e:
        pytest.skip(f"nvJPEG not available: {e}")


def _psnr(a, b):
    mse = np.mean((a.astype(np.float64) - b.astype(np.float64)) ** 2)
    return 10 * np.log10(255.0 ** 2 / max(mse, 1e-12))


def test_decoded_frames_are_close_to_their_source():
    """Camera-like frames encoded at quality 95 with 4:2:0 chroma and decoded on the device: JPEG is
    lossy, so the decoded frames are held to a PSNR against the source (> 35 dB) and the mean value of
    every channel to within 1 level."""
    j = jde()
    d = _decoder(j)
    try:
        print("backend", j.jde_decoder_backend(d))
        src = synth.frames_smooth(11, 3, 1080, 1920)
        dev = torch.from_numpy(src).cuda()
        bits = j.jde_encode_jpeg(d, dev, 3, 1920, 1080, 95, torch.cuda.current_stream())
        assert all(b[0] == 0xFF and b[1] == 0xD8 for b in bits)          # SOI marker
        out = torch.zeros_like(dev)
        j.jde_decode_jpeg(d, bits, 1920, 1080, out, torch.cuda.current_stream())
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        for i in range(3):
            p = _psnr(got[i], src[i])
            print("frame", i, "bytes", len(bits[i]), "psnr", p)
            assert p > 35.0
            assert np.all(np.abs(got[i].reshape(-1, 3).mean(0) - src[i].reshape(-1, 3).mean(0)) < 1.0)
    finally:
        j.jde_decoder_destroy(d)


def test_constant_frames_decode_to_their_colour():
    """A frame of one colour has no AC energy: it decodes to that colour within the YCbCr round trip's
    rounding (2 levels)."""
    j = jde()
    d = _decoder(j)
    try:
        cols = [(120, 60, 200), (0, 0, 0), (255, 255, 255), (17, 240, 99)]
        src = np.stack([np.broadcast_to(np.array(c, np.uint8), (192, 320, 3)) for c in cols])
        dev = torch.from_numpy(np.ascontiguousarray(src)).cuda()
        bits = j.jde_encode_jpeg(d, dev, 4, 320, 192, 100, torch.cuda.current_stream())
        out = torch.zeros_like(dev)
        j.jde_decode_jpeg(d, bits, 320, 192, out, torch.cuda.current_stream())
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(int)
        assert np.abs(got - src.astype(int)).max() <= 2
    finally:
        j.jde_decoder_destroy(d)


def test_decode_refuses_a_size_mismatch_before_any_device_work():
    j = jde()
    d = _decoder(j)
    try:
        dev = torch.from_numpy(synth.frames_smooth(2, 1, 192, 320)).cuda()
        bits = j.jde_encode_jpeg(d, dev, 1, 320, 192, 90, torch.cuda.current_stream())
        out = torch.zeros((1, 1080, 1920, 3), dtype=torch.uint8, device="cuda")
        with pytest.raises(j.JdeError):
            j.jde_decode_jpeg(d, bits, 1920, 1080, out, torch.cuda.current_stream())
        with pytest.raises(j.JdeError):
            j.jde_decode_jpeg(d, [bits[0][:2]], 320, 192, out, torch.cuda.current_stream())
        big = [bits[0]] * 5                                   # more frames than the decoder's batch
        with pytest.raises(j.JdeError):
            j.jde_decode_jpeg(d, big, 320, 192, out, torch.cuda.current_stream())
    finally:
        j.jde_decoder_destroy(d)


def test_decoded_batch_equals_frame_by_frame_decode():
    """Batched decode of four frames gives the same bytes as decoding each alone."""
    j = jde()
    d = _decoder(j)
    try:
        dev = torch.from_numpy(synth.frames_smooth(5, 4, 608, 1088)).cuda()
        bits = j.jde_encode_jpeg(d, dev, 4, 1088, 608, 90, torch.cuda.current_stream())
        out = torch.zeros_like(dev)
        j.jde_decode_jpeg(d, bits, 1088, 608, out, torch.cuda.current_stream())
        one = torch.zeros_like(dev[:1])
        torch.cuda.synchronize()
        for i in range(4):
            j.jde_decode_jpeg(d, [bits[i]], 1088, 608, one, torch.cuda.current_stream())
            torch.cuda.synchronize()
            assert torch.equal(one[0], out[i])
    finally:
        j.jde_decoder_destroy(d)
