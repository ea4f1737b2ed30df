"""Host logic of the in-tree build: concurrent build() calls (the ranks of a multi-process
launch) compile once, and the binding picks the bounds-checked library only when asked."""
import threading
import time


def test_concurrent_builds_compile_once(monkeypatch, tmp_path):
    from paper_2505_08482_gb300 import _build
    lib = tmp_path / "libpat.so"
    monkeypatch.setattr(_build, "LIBDIR", str(tmp_path))
    monkeypatch.setattr(_build, "LIB", str(lib))
    compiled = []

    def fake_compile(lib_path, bdir, verbose, extra_flags, debug):
        compiled.append(lib_path)
        time.sleep(0.3)            # long enough for the other callers to queue on the lock
        lib.write_bytes(b"x")
        return lib_path

    monkeypatch.setattr(_build, "_compile", fake_compile)
    monkeypatch.setattr(_build, "is_stale", lambda debug=False: not lib.exists())
    out = []
    threads = [threading.Thread(target=lambda: out.append(_build.build())) for _ in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert compiled == [str(lib)] and out == [str(lib)] * 4


def test_debug_library_only_on_request(monkeypatch):
    from paper_2505_08482_gb300 import _binding
    monkeypatch.delenv("PAT_DEBUG_BOUNDS", raising=False)
    assert _binding.lib_path() == _binding.LIB
    monkeypatch.setenv("PAT_DEBUG_BOUNDS", "0")
    assert _binding.lib_path() == _binding.LIB
    monkeypatch.setenv("PAT_DEBUG_BOUNDS", "1")
    assert _binding.lib_path() == _binding.LIB_DEBUG
