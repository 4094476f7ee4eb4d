"""Host logic of bench.py (CPU): the algorithmic bytes of each pass, and the
rule that a committed DRAM-traffic record counts only for the kernel sources
and the engine variant it was captured on."""
import json
import types

import bench


def _sizes(N, P, PE, Q, n_omega):
    return types.SimpleNamespace(N=N, fft_p=P, fft_e=PE, q_extent=Q, n_omega=n_omega)


def test_pass_bytes_of_the_256_cube():
    # 256^2 momenta, P = 384, PE = 256 (H = 129), Q = 256, 128 transfers
    b = bench.pass_bytes(_sizes(256, 384, 256, 256, 128))
    H = 129
    assert b["energy_fwd"] == 8 * 256 * 256 * 2 * H
    assert b["py_fwd"] == 8 * (256 * 256 * 2 * H + 256 * 384 * 2 * H)
    assert b["px_product"] == 8 * (256 * 384 * 2 * H + 256 * 384 * H) == 304349184
    assert b["py_inv"] == 8 * (256 * 384 * H + 256 * 256 * H)
    assert b["energy_inv"] == 8 * 256 * 256 * H + 4 * 256 * 256 * 128
    assert abs(sum(b.values()) / (256 * 256 * 128) - 125.0) < 1.0   # about 125 bytes per output


def test_traffic_record_needs_current_sources_and_variant(tmp_path, monkeypatch):
    rec = {"extended_256x256x256": {"px_product": {
        "kernel": "k", "variant": 4, "dram_bytes_per_launch": 123,
        "source_sha256_16": bench.source_digest(bench.PASS_FILES["px_product"])}}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    real_root = bench.ROOT
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the digest reads the kernel sources under ROOT: point it back at the repository
    monkeypatch.setattr(bench, "source_digest",
                        lambda f, _d=bench.source_digest: _with_root(_d, real_root, f))
    assert bench.recorded_traffic("px_product", "extended_256x256x256", 4) == 123
    assert bench.recorded_traffic("px_product", "extended_256x256x256", 5) is None   # another variant
    assert bench.recorded_traffic("py_inv", "extended_256x256x256", 3) is None       # no record
    rec["extended_256x256x256"]["px_product"]["source_sha256_16"] = "0" * 16          # stale sources
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    assert bench.recorded_traffic("px_product", "extended_256x256x256", 4) is None


def _with_root(digest, root, fnames):
    saved = bench.ROOT
    bench.ROOT = root
    try:
        return digest(fnames)
    finally:
        bench.ROOT = saved



def test_backward_bytes_of_the_large_workload():
    # the adjoint call at 1024^2 x 512 (P = 1536, H = 257, Q = 1024, 256
    # transfers): each pass's reads and writes counted by hand
    s = types.SimpleNamespace(N=1024, fft_p=1536, fft_e=512, q_extent=1024, n_omega=256, n_eps=512)
    H = 257
    W1, W2 = 1024 * 1024 * 2 * H, 1024 * 1536 * 2 * H          # a^ b^ along energy, along p_y
    WQ1, WQ2 = 1024 * 1024 * H, 1024 * 1536 * H                # W^ along energy, along q_y
    passes = [
        8 * W1,                                                # energy forward (write)
        8 * (W1 + W2),                                         # p_y forward
        4 * 1024 * 1024 * 256 + 8 * WQ1,                       # w along energy
        8 * (WQ1 + WQ2),                                       # w along q_y
        8 * (W2 + WQ2 + W2),                                   # products along p_x (h^, g^ over a^, b^)
        8 * (W2 + W1),                                         # p_y inverse
        8 * W1 + 4 * 1024 * 1024 * 512,                        # energy inverse, dL/dA written
    ]
    assert bench.backward_bytes(s) == sum(passes) == 57118031872
