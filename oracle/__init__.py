"""The oracle: plain, slow, obviously correct CPU evaluations of the Harris pattern pipeline.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import, call, link or run anything in this package. The CUDA library and its
Python binding never do, and this package never imports them: the two share no code.

* ``patterns``  -- the data-parallel patterns (map, zip, reduce, split, join, slide, slide2D,
                   pad_clamp, transpose, iterate) and their adjoints, on nested lists in FP64.
* ``harris``    -- the Harris pipeline as a composition of those patterns, and its reference
                   gradient by reverse mode through the pattern adjoints.
* ``cref``      -- the same pipeline as FP64 C loops, stage by stage (``harris_ref.c``), with
                   point-sampled forms for images too large for full FP64 stage arrays.
* ``mv``        -- the paper's running example (matrix-vector multiply) in both its high-level
                   and its optimised pattern form, and a row-sampled form for large matrices.
* ``corners``   -- threshold + 3x3 non-maximum suppression of R (the corner step after A5).
* ``stencil``   -- the generalised slide2D(K) + reduce stage (K x K and separable weights).
* ``harris_window`` -- the Harris pipeline with a separable K-tap window at A4.
* ``iterate_sum`` -- iterate with a shrinking body split(n) >> map(reduce(op, identity)).
* ``iterate_stencil`` -- iterate with a size-preserving body: k rounds of the clamp-padded 3x3
                   stencil.
"""
