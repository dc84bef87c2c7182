"""Host-side checks of index arithmetic the render kernel relies on (no GPU)."""
import numpy as np


def test_multiply_high_division_for_task_decoding():
    """The kernel maps a task index n to (sample, pixel slot) with n / d computed as
    umulhi(n, ceil(2^32 / d)) for block sizes d <= 32, and n itself for d = 1."""
    n = np.arange(1 << 21, dtype=np.uint64)
    for d in range(1, 33):
        m = (0xFFFFFFFF // d + 1) & 0xFFFFFFFF
        q = n if d == 1 else (n * np.uint64(m)) >> np.uint64(32)
        assert np.array_equal(q, n // d), d


def test_block_shapes_cover_images_exactly():
    """Blocks of 8, 16 or 32 pixels tile any image; ragged blocks keep every pixel slot
    inside the image."""
    shapes = {32: (8, 4), 16: (8, 2), 8: (4, 2)}
    for px, (bw, bh) in shapes.items():
        for W, H in [(1, 1), (5, 9), (17, 33), (64, 64), (257, 255)]:
            seen = np.zeros((H, W), int)
            tiles_x = (W + bw - 1) // bw
            tiles = tiles_x * ((H + bh - 1) // bh)
            for t in range(tiles):
                x0, y0 = (t % tiles_x) * bw, (t // tiles_x) * bh
                vw, vh = min(bw, W - x0), min(bh, H - y0)
                for slot in range(vw * vh):
                    x, y = x0 + slot % vw, y0 + slot // vw
                    assert x < W and y < H
                    seen[y, x] += 1
            assert np.all(seen == 1)


def test_profile_hash_ignores_comments_only():
    """bench.py reports the committed ncu counters only while the kernel sources hash as
    when they were taken; comment and blank-line edits keep the hash, code edits change it."""
    import bench
    src = 'int f(int x) {  // doubles\n    // a comment line\n\n    return 2 * x;\n}\n'
    commented = 'int f(int x) {  // twice x\n\n    // another comment\n    return 2 * x;  // result\n}\n'
    changed = 'int f(int x) {  // doubles\n    return 3 * x;\n}\n'
    assert bench._code_only(src) == bench._code_only(commented)
    assert bench._code_only(src) != bench._code_only(changed)
    files = {"paper_2211_17263_gb300/csrc/kernels.cu": src, "paper_2211_17263_gb300/csrc/internal.h": "int g;\n"}
    h1 = bench._kernel_source_sha(lambda p: files[p])
    files["paper_2211_17263_gb300/csrc/kernels.cu"] = commented
    assert bench._kernel_source_sha(lambda p: files[p]) == h1
    files["paper_2211_17263_gb300/csrc/kernels.cu"] = changed
    assert bench._kernel_source_sha(lambda p: files[p]) != h1
