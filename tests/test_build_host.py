"""CPU tests of the build's reuse rule (paper_2107_05395_gb300/build.py): the
library is reused only when the recorded hash of its inputs matches, never because
of file times."""
import os

from paper_2107_05395_gb300 import build


def test_inputs_hash_is_stable_and_depends_on_flags(monkeypatch):
    h = build.inputs_hash()
    assert h == build.inputs_hash() and len(h) == 64
    monkeypatch.setattr(build, "COMMON", build.COMMON + ["-DSOMETHING_ELSE"])
    assert build.inputs_hash() != h


def test_a_newer_library_with_a_stale_hash_is_not_reused(tmp_path, monkeypatch):
    lib = tmp_path / "libsbsolve.so"
    lib.write_bytes(b"not a library")
    monkeypatch.setattr(build, "LIB", str(lib))
    monkeypatch.setattr(build, "LIB_HASH", str(lib) + ".sha256")
    assert not build.up_to_date()  # no hash recorded
    (tmp_path / "libsbsolve.so.sha256").write_text("0" * 64 + "\n")
    os.utime(lib, (4e9, 4e9))  # far newer than every source
    assert not build.up_to_date()
    (tmp_path / "libsbsolve.so.sha256").write_text(build.inputs_hash() + "\n")
    assert build.up_to_date()
