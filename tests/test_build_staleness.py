"""The in-tree build recompiles a CUDA unit when the unit or a header is newer
than its object, or when the flags it was compiled with (VPGS_NVCC_FLAGS
included) differ from the ones recorded beside the object; otherwise it keeps
the object.  Checked with a stand-in compiler on a scratch unit (no nvcc run)."""
import os
import time
import types

from paper_2505_18992_gb300 import build as B


def _fake_compiler(calls):
    def run(cmd, capture_output=True, text=True):
        calls.append(cmd)
        out = cmd[cmd.index("-o") + 1]
        with open(out, "w") as fh:
            fh.write("obj")
        return types.SimpleNamespace(returncode=0, stderr="", stdout="")
    return run


def test_units_rebuild_on_flags_and_timestamps(tmp_path, monkeypatch):
    src = tmp_path / "unit.cu"
    src.write_text("// unit\n")
    calls = []
    monkeypatch.setattr(B, "BUILD", str(tmp_path))
    monkeypatch.setattr(B, "_headers", lambda: [])
    monkeypatch.setattr(B, "nvcc", lambda: "nvcc")
    monkeypatch.setattr(B.subprocess, "run", _fake_compiler(calls))
    monkeypatch.delenv("VPGS_NVCC_FLAGS", raising=False)

    obj = B._compile(str(src), [])
    assert len(calls) == 1 and os.path.exists(obj)
    B._compile(str(src), [])
    assert len(calls) == 1  # up to date: kept

    monkeypatch.setenv("VPGS_NVCC_FLAGS", "-DVPGS_PIX=1")
    B._compile(str(src), [])
    assert len(calls) == 2 and "-DVPGS_PIX=1" in calls[-1]  # new flags: rebuilt
    B._compile(str(src), [])
    assert len(calls) == 2

    monkeypatch.delenv("VPGS_NVCC_FLAGS")
    B._compile(str(src), [])
    assert len(calls) == 3 and "-DVPGS_PIX=1" not in calls[-1]  # back to the defaults: rebuilt

    later = time.time() + 5
    os.utime(src, (later, later))
    B._compile(str(src), [])
    assert len(calls) == 4  # the unit is newer than its object: rebuilt

