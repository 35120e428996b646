"""Host logic of the batched form's plan (no GPU): the plan file written by
the autotuner is read back as written, files for other keys or another SM
count are ignored, entries that do not exist for the keys keep the default,
and the default plan takes the smallest group whose tile holds each bin."""
import os

import pytest

CAPACITY = {"group32x16": 512, "group64x16": 1024, "group128x16": 2048, "group256x16": 4096,
            "group512x16": 8192, "group256x32": 8192, "group512x32": 16384,
            "group1024x32": 32768, "pair1024x32": 65536}


@pytest.fixture(scope="module")
def q():
    import paper_1804_10062_gb300 as q
    q.lib()
    return q


def _default(q, wide):
    out = []
    for b in range(q.QMS_BATCH_BINS):
        fits = [c for c in q.BATCH_CONFIGS if c in CAPACITY and CAPACITY[c] >= (1 << b)
                and (wide or not c.endswith("x32"))]
        out.append(min(fits, key=lambda c: (CAPACITY[c], q.BATCH_CONFIGS.index(c)))
                   if fits else "block_qms")
    return out


def test_default_plan_from_a_missing_file(q, tmp_path):
    for dtype, payload, wide in (("u32", False, True), ("u64", False, False), ("u32", True, False)):
        names, found = q.qms_batched_plan_read(str(tmp_path / "none.json"), dtype, payload, 152)
        assert not found
        assert names == _default(q, wide)


def test_plan_file_round_trip(q, tmp_path):
    names = _default(q, True)
    names[9] = "group512x16"  # bin 9 (257..512 keys): a larger group than the default
    names[14] = "block_qms"
    p = str(tmp_path / "plan.json")
    q.qms_batched_plan_write(p, names, "u32", False, 152, ns_per_key=[0.5] * q.QMS_BATCH_BINS)
    got, found = q.qms_batched_plan_read(p, "u32", False, 152)
    assert found and got == names
    # written for 152 SMs: another SM count, key width or payload ignores it
    assert q.qms_batched_plan_read(p, "u32", False, 148)[1] is False
    assert q.qms_batched_plan_read(p, "u64", False, 152)[1] is False
    assert q.qms_batched_plan_read(p, "u32", True, 152)[1] is False
    txt = open(p).read()
    assert '"sm_count": 152' in txt and '"config": "group512x16"' in txt


def test_plan_file_entries_that_do_not_fit_keep_the_default(q, tmp_path):
    p = tmp_path / "bad.json"
    lines = ['{"key_bytes": 8, "payload": 0, "sm_count": 152,', ' "bins": [']
    nb = q.QMS_BATCH_BINS
    for b in range(nb):
        cfg = "group512x32" if b == 10 else ("group32x16" if b == 12 else "group512x16")
        lines.append('  {"bin": %d, "max_len": %d, "config": "%s", "ns_per_key": 0.1}%s'
                     % (b, 1 << b, cfg, "," if b < nb - 1 else ""))
    lines.append(" ]}")
    p.write_text("\n".join(lines) + "\n")
    got, found = q.qms_batched_plan_read(str(p), "u64", False, 152)
    d = _default(q, False)
    assert found
    assert got[10] == d[10]      # 512 x 32 does not exist for 8-byte keys
    assert got[12] == d[12]      # a warp's 512 keys cannot hold 4096
    assert got[11] == "group512x16"


def test_plan_write_rejects_configurations_that_do_not_exist(q, tmp_path):
    names = _default(q, True)
    names[3] = "group512x32"
    with pytest.raises(q.QmsError):
        q.qms_batched_plan_write(str(tmp_path / "x.json"), names, "u64", True, 152)
