"""GB300-native solver for the vector-valued Allen-Cahn colour segmentation
step of Kay & Tomasi (phase field on the Gibbs simplex, Chan-Vese colour
fitting, truncated monotone multigrid on the P1 space of the pixel grid).

The compute path is the C-ABI library ``libac`` (hand-written sm_103a CUDA);
``paper_0710_0736_gb300.ac`` is its thin Python binding. Importing this
package loads nothing; importing ``.ac`` loads the library and fails loudly if
it has not been built.
"""
